"""Benchmark: SSA reaction events/s on one GB300 for the 16-bit precision modes,
against the same engine's fp64 mode.

Workload (the Schloegl configuration): the bistable Schloegl model (c1 = 3e-7,
c2 = 1e-4, c3 = 1e-3, c4 = 3.5, reservoirs A = 1e5 and B = 2e5 folded into the
rate constants), X0 = 250, 10^6 trajectories per GPU, t_end = 10, 50 evenly
spaced snapshots.  The metric counts the 16-bit modes that meet its accuracy
criterion, KS p > 0.05 of X at t_end against an independent fp64 ensemble
(10^4 trajectories each): which ones do is fixed by the workload and seeds and
stored by the oracle in tests/golden/schlogl_ks_modes.json, and the GPU run
reproduces those samples exactly (checked every run).  One timed step runs the
passing modes over the whole ensemble (`value`); the configured step of all
five 16-bit modes (mixed fp16 RN, mixed bf16 RN, uniform fp16 RN, uniform fp16
SR, uniform bf16 SR) is timed the same way beside it (`all_16bit_modes`), and
fp64 beside both.  Trajectories are independent, so N GPUs run N disjoint
trajectory-id ranges (weak scaling, no collective on the data path).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                      [--workload schlogl|tau|rdme|birth_death|telegraph|dimer|repressilator]
(--workload tau / rdme: the tau-leaping and RDME extensions, same contract;
see the section above run_ext.  birth_death / telegraph / dimer /
repressilator: the paper's other model types, see MODEL_SPECS.)
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
KS_N = 10000         # trajectories per mode in the KS criterion
OUT_SPECIES = 0b001  # snapshots store X; the reservoirs A, B are folded into c' and never change
KS_GOLDEN = os.path.join(ROOT, "tests", "golden", "schlogl_ks_modes.json")


def ks_golden():
    """The oracle's KS criterion for this workload (written by
    tests/golden/make_golden.py from the oracle alone)."""
    with open(KS_GOLDEN) as f:
        return json.load(f)


def headline_modes():
    """The configured 16-bit modes that pass the criterion."""
    passing = set(ks_golden()["passing"])
    return [m for m in MODES16 if f"{m[0]}:{m[1]}" in passing]


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
# DRAM bytes (read + write) per trajectory of one headline ensemble call, from
# one ncu count of a 4e5-trajectory call scaled per trajectory (the traffic is
# the snapshot stream and the parked records, proportional to the
# trajectories).  Valid only for the kernel source it was measured on: the key
# includes a hash of the device code, and a changed kernel reports null.
NCU_TRAFFIC_PER_TRAJ = {
    # mixed_bf16 RN (the headline kernel), 4e5 trajectories, snapshots of X only,
    # default launch shape, longest-first split: launch 1 13,282,304 R +
    # 13,166,848 W; ordering kernels 10,457,088 R; launch 2 87,435,776 R +
    # 85,055,232 W
    ("6501ac81666e509f", "mixed_bf16:rn"): (13282304 + 13166848 + 5229056 + 8448 + 5219584 + 87435776 + 85055232)
    / 400000,
}


def device_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("ssa_device.cuh", "ssa_models.h", "ssa_launch.h", "ssa_order.cu"):
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
    modes = headline_modes() or MODES16
    n_per_mode = 32 * workers * max(1, len(MODES16) // len(modes))
    for _ in range(args.warmup):
        oracle_sample(max(workers, 16), modes, workers)
    times, evs = [], []
    for _ in range(args.steps):
        e, dt = oracle_sample(n_per_mode, modes, workers)
        times.append(dt)
        evs.append(e)
    total_t, total_e = sum(times), sum(evs)
    value = total_e / total_t
    sample = (f"{n_per_mode} trajectories per mode per step (of {N_TRAJ}), trajectory ids 0..{n_per_mode - 1}, "
              f"modes {', '.join(f'{p}:{r}' for p, r in modes)}")
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
    return {"workload": f"schlogl bistable, {N_TRAJ} trajectories per GPU, t_end={T_END}, {K_SAMPLES} snapshots "
                        "of X, reservoirs folded (normalise) and not stored, int32 state; the 16-bit modes passing "
                        "KS p > 0.05 vs fp64",
            "model": "schlogl", "n_traj_per_gpu": N_TRAJ, "t_end": T_END, "n_samples": K_SAMPLES,
            "modes": [f"{p}:{r}" for p, r in (headline_modes() or MODES16)],
            "configured_modes": [f"{p}:{r}" for p, r in MODES16], "baseline_mode": "fp64",
            "max_events": MAX_EVENTS, "stored_species": "X",
            "l2": "no input reuse; each launch writes 200 MB of snapshots (> 129 MB L2)"}


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
    golden = ks_golden()
    head = headline_modes() or list(MODES16)
    modes_all = MODES16 + EXTRA_MODES + [("fp64", "rn")]
    # one output set per mode, so that the modes of a step can run concurrently
    bufs = {m: (torch.empty((K_SAMPLES, 1, N_TRAJ), dtype=torch.int32, device=dev),   # X only
                torch.empty(N_TRAJ, dtype=torch.int32, device=dev),
                torch.empty(N_TRAJ, dtype=torch.int64, device=dev),
                torch.empty(N_TRAJ, dtype=torch.float64, device=dev)) for m in modes_all}
    streams = {m: torch.cuda.Stream() for m in modes_all}
    main = torch.cuda.current_stream()

    def launch(m, seed, stream):
        out, status, nev, tfin = bufs[m]
        ssa.ensemble_run(model, N_TRAJ, x0, T_END, samples, m[0], m[1], True, seed, MAX_EVENTS, 4, out=out,
                         status=status, n_events=nev, t_final=tfin, stream=stream, traj_offset=offset,
                         out_species=OUT_SPECIES)

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

    def timed_steps(modes, record):
        if args.concurrent:
            steps = [concurrent_step(modes, SEED, record) for _ in range(args.steps)]
        else:
            steps = [sequential_step(modes, SEED, record) for _ in range(args.steps)]
        torch.cuda.synchronize()
        kernel_ms, step_ms = {}, []
        for st in steps:
            per = st[2] if args.concurrent else st
            for m, e0, e1 in per:
                kernel_ms.setdefault(m, []).append(e0.elapsed_time(e1))
            step_ms.append(st[0].elapsed_time(st[1]) if args.concurrent else
                           sum(e0.elapsed_time(e1) for _, e0, e1 in per))
        return kernel_ms, step_ms

    # warm-up (untimed): whole steps, then one sequential pass that gives each
    # mode's own rate and its samples for the KS criterion, and fp64
    for _ in range(max(0, args.warmup - 1)):
        if not args.concurrent:
            sequential_step(MODES16, SEED, None)
        else:
            concurrent_step(MODES16, SEED, None)
    rec_alone = {}
    alone = sequential_step(MODES16 + EXTRA_MODES, SEED, rec_alone)
    sequential_step([("fp64", "rn")], SEED_FP64, rec_alone)
    torch.cuda.synchronize()
    alone_ms = {m: e0.elapsed_time(e1) for m, e0, e1 in alone}

    # the KS criterion on this run's own samples (ids 0..9999 of rank 0's
    # range), against the oracle's stored values for the same trajectories
    ks_check = {}
    if rank == 0:
        ref_k = rec_alone[("fp64", "rn")][0][1][:KS_N].cpu().numpy().astype(np.int64)
        ok64 = int(ref_k.sum()) == int(round(golden["fp64_mean"] * KS_N))
        for m in MODES16 + EXTRA_MODES:
            key = f"{m[0]}:{m[1]}"
            xs = rec_alone[m][0][1][:KS_N].cpu().numpy().astype(np.int64)
            g = golden["modes"].get(key)
            p = float(sst.ks_2samp(ref_k, xs)[1])
            same = None
            if g is not None and N_TRAJ >= KS_N and rank == 0:
                same = bool(ok64 and int(xs.sum()) == g["sum_x"] and abs(p - g["ks_p"]) <= 1e-9 * max(p, 1e-300))
            ks_check[key] = {"ks_p": p, "oracle_ks_p": None if g is None else g["ks_p"], "samples_equal_oracle": same}

    # timed: K steps of the modes that meet the metric's criterion
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    rec = {}
    n0 = ssa.direct_kernel_launches()
    t0 = time.perf_counter()
    kernel_ms, step_ms = timed_steps(head, rec)
    wall = time.perf_counter() - t0
    launches_main = ssa.direct_kernel_launches() - n0
    barrier(world)
    clocks.stop()
    local_time = sum(step_ms) / 1e3
    events = {k: float(sum(float(v[0]) for v in vals)) for k, vals in rec.items()}
    local_events = sum(events.values())

    # beside it: the configured step of all five 16-bit modes, same contract
    clocks_all = ClockSampler(local)
    clocks_all.start()
    barrier(world)
    torch.cuda.synchronize()
    rec_all = {}
    n0 = ssa.direct_kernel_launches()
    kernel_all, step_all = timed_steps(MODES16, rec_all)
    launches_all = ssa.direct_kernel_launches() - n0
    barrier(world)
    clocks_all.stop()
    events_all = {k: float(sum(float(v[0]) for v in vals)) for k, vals in rec_all.items()}
    all_time = max_over_ranks(world, sum(step_all) / 1e3)
    all_events = sum_over_ranks(world, sum(events_all.values()))

    # fp64 beside it: its rate from up to three launches (6.8 s each on GB300's
    # binary64 units; the rate does not change from launch to launch)
    rec64 = {}
    steps64 = [sequential_step([("fp64", "rn")], SEED_FP64, rec64) for _ in range(min(args.steps, 3))]
    torch.cuda.synchronize()
    fp64_ms = [e0.elapsed_time(e1) for per in steps64 for _, e0, e1 in per]
    fp64_events = sum(float(v[0]) for v in rec64[("fp64", "rn")])
    fp64_rate = fp64_events / (sum(fp64_ms) / 1e3)

    # end to end through the host-buffer entry point (pinned host memory)
    h_out = torch.empty((K_SAMPLES, 1, N_TRAJ), dtype=torch.int32).pin_memory()
    h_st = torch.empty(N_TRAJ, dtype=torch.int32).pin_memory()
    h_ev = torch.empty(N_TRAJ, dtype=torch.int64).pin_memory()
    h_tf = torch.empty(N_TRAJ, dtype=torch.float64).pin_memory()
    e2e_events, e2e_time = 0.0, 0.0
    h2d = d2h = 0
    for prec, rnd in head:
        t1 = time.perf_counter()
        ssa.ensemble_run_host(model, N_TRAJ, x0, T_END, samples, prec, rnd, True, SEED, MAX_EVENTS, 4,
                              out=h_out.numpy(), status=h_st.numpy().view(np.uint32), n_events=h_ev.numpy(),
                              t_final=h_tf.numpy(), traj_offset=offset, out_species=OUT_SPECIES)
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
    for (prec, rnd), vals in rec_all.items():
        xs = vals[-1][1].cpu().numpy()
        st = vals[-1][2].cpu().numpy()
        ev_alone = float(rec_alone[(prec, rnd)][0][0])
        rate = ev_alone / (alone_ms[(prec, rnd)] / 1e3)
        modes_out[f"{prec}:{rnd}"] = {
            "events_per_s": rate, "ms_per_launch_alone": alone_ms[(prec, rnd)],
            "ms_per_launch_in_step": float(np.mean(kernel_all[(prec, rnd)])), "speedup_vs_fp64": rate / fp64_rate,
            "ks_p_vs_fp64": float(sst.ks_2samp(ref, xs)[1]),
            "ks_p_vs_fp64_n1e4": ks_check[f"{prec}:{rnd}"]["ks_p"],
            "w1_vs_fp64": float(sst.wasserstein_distance(ref, xs)),
            "mean": float(xs.mean()), "var": float(xs.var()), "frac_max_events": float(np.mean((st & 2) != 0)),
            "ops_per_event": ops_per_event(prec, rnd)}
    for prec, rnd in EXTRA_MODES:
        xs = rec_alone[(prec, rnd)][0][1].cpu().numpy()
        ev_alone = float(rec_alone[(prec, rnd)][0][0])
        rate = ev_alone / (alone_ms[(prec, rnd)] / 1e3)
        modes_out[f"{prec}:{rnd}"] = {
            "events_per_s": rate, "ms_per_launch_alone": alone_ms[(prec, rnd)], "in_step": False,
            "speedup_vs_fp64": rate / fp64_rate, "ks_p_vs_fp64": float(sst.ks_2samp(ref, xs)[1]),
            "ks_p_vs_fp64_n1e4": ks_check[f"{prec}:{rnd}"]["ks_p"],
            "w1_vs_fp64": float(sst.wasserstein_distance(ref, xs)),
            "mean": float(xs.mean()), "var": float(xs.var()), "ops_per_event": ops_per_event(prec, rnd)}
    modes_out["fp64:rn"] = {"events_per_s": fp64_rate, "ms_per_launch": float(np.mean(fp64_ms)),
                            "mean": float(ref.mean()), "var": float(ref.var())}

    sms = torch.cuda.get_device_properties(local).multi_processor_count

    def roofline(kms, evs, clk, launches):
        """ALU roofline of the step's dominant kernel (largest share): its
        operations over the whole call (with longest-first scheduling: both
        launches of the kernel and the three ordering kernels between them)."""
        dom = max(kms, key=lambda k: sum(kms[k]))
        dom_ms = float(np.mean(kms[dom]))
        dom_events = evs[dom] / args.steps
        sm_mhz = clk["sm_mhz"] or 1455.0
        peak = sms * 128 * sm_mhz * 1e6 / 1e9            # 4 schedulers x 32 lanes per SM per clock
        achieved = ops_per_event(*dom) * dom_events / (dom_ms / 1e3) / 1e9
        return {"bound": "alu", "kernel": f"ssa_kernel<schlogl,{dom[0]},{dom[1]}>",
                "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
                "traffic": traffic_per_launch(f"{dom[0]}:{dom[1]}", N_TRAJ),
                "traffic_unit": "bytes per ensemble call (all its kernels)",
                "source_hash": device_source_hash(),
                "peak_basis": f"{sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock sampled in the run)",
                "kernels_per_call": launches / (len(kms) * args.steps),
                "timed": "CUDA events around each ensemble call on its stream (every kernel of the call)",
                "snapshot_hbm_gbs": (K_SAMPLES * 1 * N_TRAJ * 4) / (dom_ms / 1e3) / 1e9}

    clk = clocks.summary()
    value = job_events / job_time
    ks_block = {"test": f"two-sample KS of X at t_end vs the independent fp64 ensemble, {KS_N} trajectories each",
                "passing_modes": [f"{p}:{r}" for p, r in head] if headline_modes() else [],
                "oracle_golden": os.path.relpath(KS_GOLDEN, ROOT),
                "samples_equal_oracle": all(v["samples_equal_oracle"] for v in ks_check.values()
                                            if v["samples_equal_oracle"] is not None),
                "per_mode": ks_check}
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * job_time / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ",".join(sorted({p.split("_")[-1] for p, _ in head})),
        "data": "synthetic", "config": config_block(),
        "gpu_launches": launches_main,
        "roofline": roofline(kernel_ms, events, clk, launches_main),
        "fp64_events_per_s": fp64_rate_job, "speedup_vs_fp64": value / fp64_rate_job,
        "ks_criterion": ks_block,
        "all_16bit_modes": {"value": all_events / all_time, "unit": "events/s",
                            "ms_per_step": 1e3 * all_time / args.steps, "steps": args.steps,
                            "gpu_launches": launches_all,
                            "speedup_vs_fp64": (all_events / all_time) / fp64_rate_job,
                            "modes": [f"{p}:{r}" for p, r in MODES16],
                            "roofline": roofline(kernel_all, events_all, clocks_all.summary(), launches_all),
                            "clocks": clocks_all.summary()},
        "modes": modes_out,
        "e2e": {"value": e2e_events / e2e_time, "unit": "events/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clk,
        "wall_s_timed": wall,
        "scheduling": {"longest_first": args.longest_first,
                       "kernels_per_call": launches_main / max(1, len(head) * args.steps)},
    }
    if world == 1 and not args.no_cpu_baseline:
        workers = os.cpu_count() or 1
        n_per_mode = 32 * workers * max(1, len(MODES16) // len(head))
        e, dt = oracle_sample(n_per_mode, head, workers)
        line["cpu_baseline"] = {"value": e / dt, "unit": "events/s", "cores": workers, "kind": "oracle",
                                "sample": f"{n_per_mode} trajectories per mode (ids 0..{n_per_mode - 1}) of the "
                                          f"same workload and modes, one process per core"}
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
    ("3c23ba7ec014e430", "tau", "fp32:rn"): {"warp_inst": 6.2743, "dram_bytes": 0.01304},
    ("3c23ba7ec014e430", "tau", "mixed_f16:rn"): {"warp_inst": 6.3621, "dram_bytes": 0.01402},
    ("3c23ba7ec014e430", "tau", "mixed_bf16:rn"): {"warp_inst": 6.2441, "dram_bytes": 0.01384},
    ("3c23ba7ec014e430", "tau", "uniform_f16:sr"): {"warp_inst": 6.5411, "dram_bytes": 0.01409},
    ("3c23ba7ec014e430", "tau", "uniform_bf16:sr"): {"warp_inst": 6.4396, "dram_bytes": 0.01364},
    # rdme, 32768 lattices, one launch per mode
    ("1a5bb4191f753f15", "rdme", "fp32:rn"): {"warp_inst": 30.1687, "dram_bytes": 0.00014},
    ("1a5bb4191f753f15", "rdme", "mixed_f16:rn"): {"warp_inst": 32.4930, "dram_bytes": 0.00017},
    ("1a5bb4191f753f15", "rdme", "mixed_bf16:rn"): {"warp_inst": 32.5187, "dram_bytes": 0.00063},
    ("1a5bb4191f753f15", "rdme", "mixed_f16:sr"): {"warp_inst": 43.9234, "dram_bytes": 0.00106},
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


# ============================================ the paper's five model types
# --workload birth_death | telegraph | dimer | repressilator: the direct-method
# step on each of the other model types of the paper (Sec. 4.1, 4.3-4.5; the
# Schloegl model is the default line), same contract: one step = the five
# configured 16-bit modes over the whole ensemble, fp64 beside it on a smaller
# ensemble, KS p / W1 of the reported species at t_end per mode against fp64
# (10^4 trajectories each), e2e through the host-buffer entry point, the
# oracle as cpu_baseline.  Parameters: birth-death k = 10, gamma = 0.1, X0 = 0,
# t_end = 100 (the parity configuration's model, scaled to 4e6 trajectories
# for throughput); telegraph at the geometric centre of the batched sweep's
# ranges (kon = koff = 0.5, km = sqrt(5 * 100), gamma = 1), dimer k1 = 1e-3,
# k2 = 0.1, M0 = 300, and the repressilator (alpha0 = 0.216, alpha = 216,
# n = 2, beta = 5, protein decay 5), t_end = 200 for all three.  101 evenly
# spaced snapshots.  Roofline: the ALU operation count per event derived from
# the model's structure (the accounting of ops_per_event, applied per
# reaction), against SMs x 128 lanes x the sampled clock.
MODEL_SPECS = {
    "birth_death": {"ctor": lambda: P.birth_death(10.0, 0.1), "x0": [0], "t_end": 100.0, "n": 4_000_000,
                    "n64": 200_000, "species": 0, "cap": 10**6, "label": "birth-death k=10, gamma=0.1, X0=0"},
    "telegraph": {"ctor": lambda: P.telegraph(0.5, 0.5, float(np.sqrt(500.0)), 1.0), "x0": list(P.TELEGRAPH_X0),
                  "t_end": 200.0, "n": 2_000_000, "n64": 100_000, "species": 2, "cap": 10**6,
                  "label": "telegraph kon=koff=0.5, km=22.36, gamma=1, gene off, no mRNA"},
    "dimer": {"ctor": lambda: P.dimer(1e-3, 0.1), "x0": list(P.dimer_x0(300)), "t_end": 200.0, "n": 2_000_000,
              "n64": 100_000, "species": 1, "cap": 10**6, "label": "dimerisation k1=1e-3, k2=0.1, M0=300"},
    "repressilator": {"ctor": lambda: P.repressilator(), "x0": list(P.REPRESSILATOR_X0), "t_end": 200.0,
                      "n": 500_000, "n64": 10_000, "species": 3, "cap": 4 * 10**6,
                      "label": "repressilator alpha0=0.216, alpha=216, n=2, beta=5, protein decay 5, P_A(0)=5"},
}
MODEL_K = 101


def model_ops_per_event(md, prec, rnd, normalise=False):
    """Algorithmic 32-bit operations per event for a model's structure, with
    the per-item costs of ops_per_event (Philox half a block per step plus
    uniform scaling, log, the tau / target / clock operations, 3 per
    mass-action factor, h + 3 per Hill term, M - 1 sums, selection, update and
    loop; 16-bit conversions, uniform-mode roundings and SR Philox blocks)."""
    order = np.asarray(md["order"])
    M, N = order.shape
    law = np.asarray(md.get("law") if md.get("law") is not None else np.zeros(M), dtype=int)
    const = np.asarray(md.get("constant") if md.get("constant") is not None else np.zeros(N), dtype=bool)
    hill = md.get("hill")
    factors, hill_ops, chain16 = 0, 0, 0
    for j in range(M):
        if law[j] == 1:
            h = int(hill[j][2])
            hill_ops += h + 3
            chain16 += h + 3
        else:
            f = int(sum(order[j][i] for i in range(N) if not (normalise and const[i])))
            factors += f
            chain16 += 2 * f
    n_update = int(sum(1 for i in range(N) if not const[i])) + 1
    ops = 100 * 0.5 + 8 + 25 + 3 + 3 * factors + hill_ops + (M - 1) + M + 2 + n_update + 1 + 4
    if prec.startswith(("mixed", "uniform")):
        ops += chain16                      # one conversion per rounded chain operation
    if prec.startswith("uniform"):
        ops += (M - 1 + 5) * 2
    if rnd == "sr":
        n_sr = chain16 + (M - 1 + 5 if prec.startswith("uniform") else 0)
        ops += 100 * ((n_sr + 7) // 8)
    if rnd == "sra":
        ops += 100 * ((M + 7) // 8)
    return float(ops)


def model_spec(workload, n_traj=None):
    sp = dict(MODEL_SPECS[workload])
    sp["model"] = sp["ctor"]()
    if n_traj:
        sp["n"] = n_traj
        sp["n64"] = min(sp["n64"], n_traj)
    sp["samples"] = P.even_samples(sp["t_end"], MODEL_K)
    sp["metric"] = f"SSA reaction events/s on 1 GB300 ({workload.replace('_', '-')}), 16-bit modes vs fp64"
    sp["config"] = {"workload": f"{sp['label']}, {sp['n']} trajectories per GPU, t_end={sp['t_end']}, "
                                f"{MODEL_K} snapshots, int32 state",
                    "model": workload, "n_traj_per_gpu": sp["n"], "t_end": sp["t_end"], "n_samples": MODEL_K,
                    "modes": [f"{p}:{r}" for p, r in MODES16], "baseline_mode": "fp64",
                    "max_events": sp["cap"],
                    "l2": "no input reuse; each launch writes its snapshot stream "
                          f"({MODEL_K * len(sp['x0']) * 4 * sp['n'] / 1e6:.0f} MB, > 129 MB L2)"}
    return sp


def models_oracle_sample(sp, modes, n_per_mode, workers):
    import oracle
    events = 0
    t0 = time.perf_counter()
    for prec, rnd in modes:
        r = oracle.run_parallel(sp["model"], sp["x0"], n_per_mode, sp["t_end"], sp["samples"], workers=workers,
                                precision=prec, rounding=rnd, normalise=False, seed=SEED, max_events=sp["cap"])
        events += int(r["n_events"].sum())
    return events, time.perf_counter() - t0


def models_oracle_n(workload, workers):
    per_traj = {"birth_death": 2e3, "telegraph": 8e3, "dimer": 4e3, "repressilator": 2.6e5}[workload]
    # about 10 s of the oracle on all host cores for the five modes
    return max(workers, int(10 * 2.0e6 * workers / per_traj / len(MODES16)) // workers * workers)


def run_models_reference(args, world, rank, workload):
    if rank != 0:
        return
    sp = model_spec(workload)
    workers = os.cpu_count() or 1
    n = models_oracle_n(workload, workers)
    for _ in range(args.warmup):
        models_oracle_sample(sp, MODES16, workers, workers)
    times, evs = [], []
    for _ in range(args.steps):
        e, dt = models_oracle_sample(sp, MODES16, n, workers)
        times.append(dt)
        evs.append(e)
    value = sum(evs) / sum(times)
    sample = f"{n} trajectories per 16-bit mode per step (of {sp['n']}), ids 0..{n - 1}"
    print(json.dumps({
        "impl": "reference", "metric": sp["metric"], "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16,bf16",
        "data": "synthetic", "config": sp["config"],
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": workers, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def run_models(args, world, rank, local, workload):
    import torch
    from scipy import stats as sst
    from paper_2605_00479_gb300 import ssa

    torch.cuda.set_device(local)
    ssa.lib()
    sp = model_spec(workload, args.n_traj)
    model = ssa.Model.from_dict(sp["model"])
    n, n64 = sp["n"], sp["n64"]
    offset = rank * n
    main = torch.cuda.current_stream()
    K, N = len(sp["samples"]), model.N
    x0 = np.asarray(sp["x0"], dtype=np.int32)

    def buffers(count):
        return (torch.empty((K, N, count), dtype=torch.int32, device="cuda"),
                torch.empty(count, dtype=torch.int32, device="cuda"),
                torch.empty(count, dtype=torch.int64, device="cuda"),
                torch.empty(count, dtype=torch.float64, device="cuda"))

    bufs = {m: buffers(n) for m in MODES16}
    bufs[("fp64", "rn")] = buffers(n64)

    def step(modes, seed, count):
        per = []
        for m in modes:
            out, st, ev, tf = bufs[m]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            ssa.ensemble_run(model, count, x0, sp["t_end"], sp["samples"], m[0], m[1], False, seed, sp["cap"], 4,
                             out=out, status=st, n_events=ev, t_final=tf, stream=main, traj_offset=offset)
            e1.record(main)
            per.append((m, e0, e1))
        torch.cuda.synchronize()
        res = {}
        for m, e0, e1 in per:
            out, st, ev, _ = bufs[m]
            res[m] = (e0.elapsed_time(e1), float(ev[:count].double().sum()),
                      out[-1, sp["species"], :count].cpu().numpy(), int(((st[:count] & 0xB) != 0).sum().item()))
        return res

    for _ in range(args.warmup):
        step(MODES16, SEED, n)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    n_l0 = ssa.direct_kernel_launches()
    t0 = time.perf_counter()
    steps = [step(MODES16, SEED, n) for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    launches = ssa.direct_kernel_launches() - n_l0
    barrier(world)
    clocks.stop()
    local_time = sum(v[0] for st in steps for v in st.values()) / 1e3
    local_events = sum(v[1] for st in steps for v in st.values())
    job_time = max_over_ranks(world, local_time)
    job_events = sum_over_ranks(world, local_events)

    step([("fp64", "rn")], SEED + 1, n64)
    r64 = step([("fp64", "rn")], SEED + 1, n64)[("fp64", "rn")]
    fp64_rate = r64[1] / (r64[0] / 1e3)

    # end to end through the host-buffer entry point (pinned host memory); one
    # untimed call first (the entry point's staging memory pool grows once per
    # process)
    h = [torch.empty(v.shape, dtype=v.dtype).pin_memory() for v in bufs[MODES16[0]]]
    ssa.ensemble_run_host(model, n, x0, sp["t_end"], sp["samples"], MODES16[0][0], MODES16[0][1], False, SEED,
                          sp["cap"], 4, out=h[0].numpy(), status=h[1].numpy().view(np.uint32), n_events=h[2].numpy(),
                          t_final=h[3].numpy(), traj_offset=offset)
    e2e_events, e2e_time = 0.0, 0.0
    h2d = len(MODES16) * (x0.nbytes + np.asarray(sp["samples"]).nbytes)          # per step
    d2h = len(MODES16) * sum(v.numel() * v.element_size() for v in h)
    e2e_ms = {f"{p}:{r}": [] for p, r in MODES16}
    for _ in range(args.steps):                                  # the same steps as the device timing
        for prec, rnd in MODES16:
            t1 = time.perf_counter()
            ssa.ensemble_run_host(model, n, x0, sp["t_end"], sp["samples"], prec, rnd, False, SEED, sp["cap"], 4,
                                  out=h[0].numpy(), status=h[1].numpy().view(np.uint32), n_events=h[2].numpy(),
                                  t_final=h[3].numpy(), traj_offset=offset)
            dt = time.perf_counter() - t1
            e2e_time += dt
            e2e_ms[f"{prec}:{rnd}"].append(round(1e3 * dt, 2))
            e2e_events += float(h[2].numpy().sum())
    e2e_time = max_over_ranks(world, e2e_time)
    e2e_events = sum_over_ranks(world, e2e_events)
    if rank != 0:
        return

    ref = r64[2]
    ref_k = ref[:KS_N]
    modes_out = {"fp64:rn": {"events_per_s": fp64_rate, "ms_per_launch": r64[0], "n_traj": n64,
                             "mean": float(ref.mean()), "var": float(ref.var())}}
    clk = clocks.summary()
    sm_mhz = clk["sm_mhz"] or 1455.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * 128 * sm_mhz * 1e6 / 1e9
    for m in MODES16:
        ms = [st[m][0] for st in steps]
        ev = sum(st[m][1] for st in steps)
        rate = ev / (sum(ms) / 1e3)
        xs = steps[-1][m][2]
        opsv = model_ops_per_event(sp["model"], *m)
        modes_out[f"{m[0]}:{m[1]}"] = {
            "events_per_s": rate, "ms_per_launch": float(np.mean(ms)), "events_per_launch": steps[-1][m][1],
            "speedup_vs_fp64": rate / fp64_rate, "ks_p_vs_fp64_n1e4": float(sst.ks_2samp(ref_k, xs[:KS_N])[1]),
            "w1_vs_fp64": float(sst.wasserstein_distance(ref, xs)), "mean": float(xs.mean()),
            "var": float(xs.var()), "stopped": steps[-1][m][3], "ops_per_event": opsv,
            "alu_frac": opsv * rate / 1e9 / peak}
    dom = max(MODES16, key=lambda m: sum(st[m][0] for st in steps))
    dom_ms = float(np.mean([st[dom][0] for st in steps]))
    dom_events = float(np.mean([st[dom][1] for st in steps]))
    achieved = model_ops_per_event(sp["model"], *dom) * dom_events / (dom_ms / 1e3) / 1e9
    value = job_events / job_time
    line = {
        "metric": sp["metric"], "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * job_time / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16,bf16", "data": "synthetic", "config": sp["config"],
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": f"ssa_kernel<{workload},{dom[0]},{dom[1]}>", "achieved": achieved,
                     "peak": peak, "unit": "Gop/s", "frac": achieved / peak, "traffic": None,
                     "traffic_unit": "bytes per launch", "source_hash": device_source_hash(),
                     "peak_basis": f"{sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock sampled in the run)",
                     "ops_per_event": model_ops_per_event(sp["model"], *dom),
                     "snapshot_hbm_gbs": (K * N * n * 4) / (dom_ms / 1e3) / 1e9},
        "fp64_events_per_s": fp64_rate, "speedup_vs_fp64": value / fp64_rate,
        "ks_criterion": {"test": f"two-sample KS of species {sp['species']} at t_end vs an independent fp64 "
                                 f"ensemble, {KS_N} trajectories each",
                         "passing_modes": [f"{p}:{r}" for p, r in MODES16
                                           if modes_out[f"{p}:{r}"]["ks_p_vs_fp64_n1e4"] > 0.05]},
        "modes": modes_out,
        "e2e": {"value": e2e_events / e2e_time, "unit": "events/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_call": e2e_ms},
        "clocks": clk, "wall_s_timed": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        workers = os.cpu_count() or 1
        nn = models_oracle_n(workload, workers)
        e, dt = models_oracle_sample(sp, MODES16, nn, workers)
        line["cpu_baseline"] = {"value": e / dt, "unit": "events/s", "cores": workers, "kind": "oracle",
                                "sample": f"{nn} trajectories per mode (ids 0..{nn - 1}) of the same workload, "
                                          "one process per core"}
    print(json.dumps(line), flush=True)


# ======================================== batched sweep and the scale run
# --workload batch: the heterogeneous batched configuration -- telegraph
# (kon, koff log-uniform in [0.05, 5], km in [5, 100], gamma 1), dimerisation
# (k1, k2 log-uniform in [x0.5, x2] around 1e-3 and 0.1; M0 = 300) and
# repressilator (alpha, beta log-uniform in [x0.5, x2] around 216 and 5)
# sweeps of 10^4 parameter sets x 256 trajectories each, t_end = 200, one
# snapshot at t_end, all three models in ONE persistent launch replayed from a
# CUDA graph, launch shape from the project's autotuner (run in warm-up); one
# step = mixed fp16 RN and uniform bf16 SR.
# --workload scale: the repressilator throughput / memory run -- 10^7
# trajectories per GPU to t_end = 1000 with 200 snapshots streamed to HBM
# (48 GB int32 / 24 GB int16), state stored int32 and int16, propensities
# fp16 (mixed) and fp32; fp64 beside it on 2e4 trajectories (GB300's binary64
# rate puts the full ensemble at over an hour).  One step runs the four
# (precision, storage) combinations over the whole ensemble, so a step takes
# minutes; warm-up steps run 10^5 trajectories.  e2e is taken on a 10^6
# trajectory slice (results written straight into page-locked host memory).
BATCH_SETS, BATCH_TRAJ, BATCH_T_END = 10_000, 256, 200.0
BATCH_MODES = [("mixed_f16", "rn"), ("uniform_bf16", "sr")]
SCALE_N, SCALE_T_END, SCALE_K, SCALE_N64, SCALE_WARM_N, SCALE_E2E_N = 10_000_000, 1000.0, 200, 20_000, 100_000, \
    1_000_000
SCALE_RUNS = [("mixed_f16", 4), ("mixed_f16", 2), ("fp32", 4), ("fp32", 2)]

# warp instructions per event from one ncu count (smsp__inst_executed.sum over
# the launch / events), keyed by (device-source hash, workload, mode): the
# issue-rate fraction of those kernels; null once the kernel source changes
NCU_INST_PER_EVENT = {}


def batch_groups(ssa=None, seed=3):
    """The batched sweep's groups (with engine models when `ssa` is given)."""
    tel, dm, rp = P.telegraph(), P.dimer(), P.repressilator()
    tr = P.telegraph_sweep(BATCH_SETS, seed=seed)
    dr = P.dimer_sweep(BATCH_SETS, seed=seed + 1)
    rr, rh = P.repressilator_sweep(BATCH_SETS, seed=seed + 2)
    n = BATCH_SETS * BATCH_TRAJ
    specs = [("repressilator", rp, P.REPRESSILATOR_X0, rr, rh[:, :, :2]), ("telegraph", tel, P.TELEGRAPH_X0, tr, None),
             ("dimer", dm, P.dimer_x0(300), dr, None)]
    groups = []
    for g, (name, md, x0, rates, hill) in enumerate(specs):
        groups.append({"name": name, "dict": md, "model": ssa.Model.from_dict(md) if ssa is not None else None,
                       "x0": np.tile(x0, (BATCH_SETS, 1)), "rates": rates, "hill": hill,
                       "traj_per_set": BATCH_TRAJ, "traj_offset": g * n})
    return groups


def batch_oracle_sample(groups, modes=BATCH_MODES):
    """The oracle on a bounded sample of the batched sweep: trajectory 0 of the
    first parameter sets of each model (fewer repressilator sets, whose
    trajectories are ~50x longer), every mode, one process per core."""
    import oracle
    workers = os.cpu_count() or 1
    e_tot, t_tot = 0, 0.0
    for prec, rnd in modes:
        for G in groups:
            sets = workers if G["name"] == "repressilator" else 8 * workers
            jobs_md = []
            for q in range(sets):
                md = dict(G["dict"])
                md["rate"] = G["rates"][q]
                if G["hill"] is not None:
                    h = np.array(md["hill"], dtype=np.float64, copy=True)
                    h[:, :2] = G["hill"][q]
                    md["hill"] = h
                jobs_md.append(md)
            t1 = time.perf_counter()
            for q, md in enumerate(jobs_md):
                r = oracle.run(md, G["x0"][q], 1, BATCH_T_END, [BATCH_T_END], prec, rnd, False, SEED, 10**7,
                               g0=G["traj_offset"] + q * BATCH_TRAJ)
                e_tot += int(r["n_events"].sum())
            t_tot += time.perf_counter() - t1
    return e_tot, t_tot, (f"trajectory 0 of the first {8 * workers} telegraph and dimer sets and {workers} "
                          "repressilator sets, both modes, one process")


def scale_oracle_sample():
    import oracle
    workers = os.cpu_count() or 1
    md = P.repressilator()
    samples = P.even_samples(SCALE_T_END, SCALE_K)
    t1 = time.perf_counter()
    r = oracle.run_parallel(md, P.REPRESSILATOR_X0, workers, SCALE_T_END, samples, workers=workers,
                            precision="mixed_f16", rounding="rn", seed=SEED, max_events=10**9, state_bytes=2)
    dt = time.perf_counter() - t1
    return float(r["n_events"].sum()), dt, (f"{workers} trajectories (ids 0..{workers - 1}), mixed fp16, int16 "
                                            "state, one process per core")


def run_batch_scale_reference(args, world, rank, workload):
    if rank != 0:
        return
    times, evs = [], []
    for i in range(args.warmup + args.steps):
        if workload == "batch":
            e, dt, sample = batch_oracle_sample(batch_groups())
        else:
            e, dt, sample = scale_oracle_sample()
        if i >= args.warmup:
            times.append(dt)
            evs.append(e)
    value = sum(evs) / sum(times)
    print(json.dumps({
        "impl": "reference", "metric": f"SSA reaction events/s ({workload} workload)", "value": value,
        "unit": "events/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16,bf16", "data": "synthetic", "config": {"workload": workload},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


def run_batch(args, world, rank, local):
    import torch
    from paper_2605_00479_gb300 import ssa

    torch.cuda.set_device(local)
    ssa.lib()
    groups = batch_groups(ssa)
    for G in groups:
        G["traj_offset"] += rank * 3 * BATCH_SETS * BATCH_TRAJ
    s = torch.cuda.Stream()
    batches, tune = {}, {}
    for prec, rnd in BATCH_MODES:
        batches[(prec, rnd)] = ssa.Batch(groups, BATCH_T_END, [BATCH_T_END], prec, rnd, seed=SEED,
                                         max_events=10**7)
        tune[(prec, rnd)] = batches[(prec, rnd)].autotune(s)

    def step():
        per = []
        for m in BATCH_MODES:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            batches[m].launch(s)
            e1.record(s)
            per.append((m, e0, e1))
        s.synchronize()
        return {m: (e0.elapsed_time(e1), [float(o["n_events"].double().sum()) for o in batches[m].outputs],
                    sum(int((o["status"] != 0).sum()) for o in batches[m].outputs)) for m, e0, e1 in per}

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    n_l0 = ssa.direct_kernel_launches()
    t0 = time.perf_counter()
    steps = [step() for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    launches = ssa.direct_kernel_launches() - n_l0
    barrier(world)
    clocks.stop()
    local_time = sum(v[0] for st in steps for v in st.values()) / 1e3
    local_events = sum(sum(v[1]) for st in steps for v in st.values())
    job_time = max_over_ranks(world, local_time)
    job_events = sum_over_ranks(world, local_events)

    # end to end: create (per-set tables uploaded from the host) + launch, results
    # written into page-locked host memory by the kernel
    e2e_events, e2e_time, h2d, d2h = 0.0, 0.0, 0, 0
    for prec, rnd in BATCH_MODES:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        t = tune[(prec, rnd)]
        ssa.set_launch_config(t["threads_per_block"], t["blocks_per_sm"], t["slice_pairs"])   # the tuned shape
        try:
            b = ssa.Batch(groups, BATCH_T_END, [BATCH_T_END], prec, rnd, seed=SEED, max_events=10**7,
                          host_outputs=True)
        finally:
            ssa.set_launch_config()
        b.launch(None)
        torch.cuda.synchronize()
        e2e_time += time.perf_counter() - t1
        e2e_events += sum(float(o["n_events"].double().sum()) for o in b.outputs)
        h2d += sum(G["x0"].nbytes + G["rates"].nbytes + (0 if G["hill"] is None else G["hill"].nbytes)
                   for G in groups)
        d2h += sum(v.numel() * v.element_size() for o in b.outputs for v in o.values())
        b.close()
    e2e_time = max_over_ranks(world, e2e_time)
    e2e_events = sum_over_ranks(world, e2e_events)
    if rank != 0:
        return
    clk = clocks.summary()
    sm_mhz = clk["sm_mhz"] or 1455.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * 128 * sm_mhz * 1e6 / 1e9
    modes_out = {}
    for m in BATCH_MODES:
        ms = [st[m][0] for st in steps]
        ev_g = [sum(st[m][1][g] for st in steps) for g in range(3)]
        ops = sum(model_ops_per_event(G["dict"], *m) * e for G, e in zip(groups, ev_g))
        modes_out[f"{m[0]}:{m[1]}"] = {
            "events_per_s": sum(ev_g) / (sum(ms) / 1e3), "ms_per_launch": float(np.mean(ms)),
            "events_per_model": {G["name"]: e / args.steps for G, e in zip(groups, ev_g)},
            "alu_frac": ops / (sum(ms) / 1e3) / 1e9 / peak, "autotune": tune[m],
            "nonzero_status": steps[-1][m][2]}
    dom = max(BATCH_MODES, key=lambda m: sum(st[m][0] for st in steps))
    dom_ms = sum(st[dom][0] for st in steps)
    dom_ops = sum(model_ops_per_event(G["dict"], *dom) * sum(st[dom][1][g] for st in steps)
                  for g, G in enumerate(groups))
    achieved = dom_ops / (dom_ms / 1e3) / 1e9
    value = job_events / job_time
    n_tot = 3 * BATCH_SETS * BATCH_TRAJ
    line = {
        "metric": "SSA reaction events/s on 1 GB300 (batched heterogeneous sweep, one persistent launch)",
        "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * job_time / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16,bf16", "data": "synthetic",
        "config": {"workload": f"batched sweep: telegraph + dimerisation + repressilator, {BATCH_SETS} parameter "
                               f"sets x {BATCH_TRAJ} trajectories each per GPU ({n_tot} trajectories), "
                               f"t_end={BATCH_T_END}, snapshot at t_end, one persistent launch per mode",
                   "models": ["repressilator", "telegraph", "dimer"], "n_traj_per_gpu": n_tot,
                   "t_end": BATCH_T_END, "n_samples": 1, "modes": [f"{p}:{r}" for p, r in BATCH_MODES],
                   "l2": "each launch simulates 7.7e11 events with state in registers; no input reuse"},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": f"ssa_batch_kernel<{dom[0]},{dom[1]},telegraph,dimer,repressilator>",
                     "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak, "traffic": None,
                     "traffic_unit": "bytes per launch", "source_hash": device_source_hash(),
                     "peak_basis": f"{sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock sampled in the run)",
                     "ops_basis": "per-model structural op count x that model's events"},
        "modes": modes_out,
        "e2e": {"value": e2e_events / e2e_time, "unit": "events/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "note": "ssa_batch_create (per-set tables uploaded) + launch per mode, results in page-locked "
                        "host memory"},
        "clocks": clk, "wall_s_timed": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        e, dt, sample = batch_oracle_sample(groups)
        line["cpu_baseline"] = {"value": e / dt, "unit": "events/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": sample}
    print(json.dumps(line), flush=True)


def run_scale(args, world, rank, local):
    import torch
    from paper_2605_00479_gb300 import ssa

    torch.cuda.set_device(local)
    ssa.lib()
    md = P.repressilator()
    model = ssa.Model.from_dict(md)
    x0 = P.REPRESSILATOR_X0
    n = args.n_traj or SCALE_N
    samples = P.even_samples(SCALE_T_END, SCALE_K)
    offset = rank * n
    free0 = torch.cuda.mem_get_info()[0]
    outs = {sb: torch.empty((SCALE_K, model.N, n), dtype=torch.int16 if sb == 2 else torch.int32, device="cuda")
            for sb in (4, 2)}
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ev = torch.empty(n, dtype=torch.int64, device="cuda")
    main = torch.cuda.current_stream()

    def launch(prec, sb, count, seed=SEED):
        o = outs[sb][:, :, :count] if count == n else torch.empty((SCALE_K, model.N, count), dtype=outs[sb].dtype,
                                                                    device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        ssa.ensemble_run(model, count, x0, SCALE_T_END, samples, prec, "rn", False, seed, 10**9, sb, out=o,
                         status=st[:count], n_events=ev[:count], t_final=None, with_t_final=False, stream=main,
                         traj_offset=offset)
        e1.record(main)
        torch.cuda.synchronize()
        return (e0.elapsed_time(e1), float(ev[:count].double().sum()),
                int(((st[:count] & 4) != 0).sum().item()), int(o.abs().max().item()))

    for _ in range(args.warmup):
        for prec, sb in SCALE_RUNS:
            launch(prec, sb, min(SCALE_WARM_N, n))
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    n_l0 = ssa.direct_kernel_launches()
    t0 = time.perf_counter()
    steps = [{(prec, sb): launch(prec, sb, n) for prec, sb in SCALE_RUNS} for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    launches = ssa.direct_kernel_launches() - n_l0
    barrier(world)
    clocks.stop()
    local_time = sum(v[0] for stp in steps for v in stp.values()) / 1e3
    local_events = sum(v[1] for stp in steps for v in stp.values())
    job_time = max_over_ranks(world, local_time)
    job_events = sum_over_ranks(world, local_events)
    n64 = min(SCALE_N64, n)
    fp64 = {sb: launch("fp64", sb, n64) for sb in (4, 2)}
    # end to end on a slice: page-locked host outputs written by the kernel
    ne = min(SCALE_E2E_N, n)
    h = [torch.empty((SCALE_K, model.N, ne), dtype=torch.int16).pin_memory(),
         torch.empty(ne, dtype=torch.int32).pin_memory(), torch.empty(ne, dtype=torch.int64).pin_memory(),
         torch.empty(ne, dtype=torch.float64).pin_memory()]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ssa.ensemble_run_host(model, ne, x0, SCALE_T_END, samples, "mixed_f16", "rn", False, SEED, 10**9, 2,
                          out=h[0].numpy(), status=h[1].numpy().view(np.uint32), n_events=h[2].numpy(),
                          t_final=h[3].numpy(), traj_offset=offset)
    e2e_t = time.perf_counter() - t1
    e2e_ev = float(h[2].numpy().sum())
    if rank != 0:
        return
    clk = clocks.summary()
    sm_mhz = clk["sm_mhz"] or 1455.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * 128 * sm_mhz * 1e6 / 1e9
    peak_issue = sms * 4 * sm_mhz * 1e6 / 1e9
    runs = {}
    for prec, sb in SCALE_RUNS + [("fp64", 4), ("fp64", 2)]:
        if prec == "fp64":
            ms, evs, flags, mx = fp64[sb]
            count = n64
        else:
            ms = float(np.mean([stp[(prec, sb)][0] for stp in steps]))
            evs = float(np.mean([stp[(prec, sb)][1] for stp in steps]))
            flags, mx = steps[-1][(prec, sb)][2], steps[-1][(prec, sb)][3]
            count = n
        rate = evs / (ms / 1e3)
        opsv = model_ops_per_event(md, prec, "rn")
        inst = NCU_INST_PER_EVENT.get((device_source_hash(), "scale", f"{prec}:rn"))
        runs[f"{prec}:int{8 * sb}"] = {
            "n_traj": count, "events": evs, "seconds": ms / 1e3, "events_per_s": rate,
            "bytes_per_traj": SCALE_K * model.N * sb, "snapshot_hbm_gbs": SCALE_K * model.N * sb * count / (ms / 1e3) / 1e9,
            "alu_frac": opsv * rate / 1e9 / peak, "ops_per_event": opsv,
            "issue_frac": None if inst is None else inst * rate / 1e9 / peak_issue,
            "state_range_flags": flags, "max_abs_state": mx}
    dom = max(SCALE_RUNS, key=lambda r: sum(stp[r][0] for stp in steps))
    dom_ms = float(np.mean([stp[dom][0] for stp in steps]))
    dom_ev = float(np.mean([stp[dom][1] for stp in steps]))
    achieved = model_ops_per_event(md, dom[0], "rn") * dom_ev / (dom_ms / 1e3) / 1e9
    value = job_events / job_time
    line = {
        "metric": "SSA reaction events/s on 1 GB300 (repressilator scale run, int16/int32 state, fp16/fp32)",
        "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * job_time / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16,f32", "data": "synthetic",
        "config": {"workload": f"repressilator, {n} trajectories per GPU, t_end={SCALE_T_END}, {SCALE_K} snapshots "
                               "streamed to HBM, state stored int32 and int16, propensities fp16 (mixed) and fp32",
                   "model": "repressilator", "n_traj_per_gpu": n, "t_end": SCALE_T_END, "n_samples": SCALE_K,
                   "runs": [f"{p}:int{8 * sb}" for p, sb in SCALE_RUNS], "fp64_subsample": n64,
                   "hbm_free_gb_before": free0 / 1e9,
                   "l2": f"each launch writes {SCALE_K * 6 * n * 2 / 1e9:.0f}-{SCALE_K * 6 * n * 4 / 1e9:.0f} GB of "
                         "snapshots (> 129 MB L2)"},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": f"ssa_kernel<repressilator,{dom[0]},rn>", "achieved": achieved,
                     "peak": peak, "unit": "Gop/s", "frac": achieved / peak, "traffic": None,
                     "traffic_unit": "bytes per launch", "source_hash": device_source_hash(),
                     "peak_basis": f"{sms} SMs x 128 lanes x {sm_mhz:.0f} MHz (median SM clock sampled in the run)"},
        "runs": runs,
        "e2e": {"value": e2e_ev / e2e_t, "unit": "events/s", "h2d_bytes_per_step": int(x0.nbytes + samples.nbytes),
                "d2h_bytes_per_step": int(sum(v.numel() * v.element_size() for v in h)),
                "note": f"mixed fp16, int16 state, {ne} trajectories, results written into page-locked host memory"},
        "clocks": clk, "wall_s_timed": wall,
    }
    if world == 1 and not args.no_cpu_baseline:
        e, dt, sample = scale_oracle_sample()
        line["cpu_baseline"] = {"value": e / dt, "unit": "events/s", "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": sample}
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
    ap.add_argument("--workload", choices=["schlogl", "tau", "rdme", "batch", "scale"] + list(MODEL_SPECS),
                    default="schlogl",
                    help="schlogl: the direct-method benchmark (default); tau: tau-leaping; rdme: spatial RDME; "
                         "birth_death / telegraph / dimer / repressilator: the other model types")
    ap.add_argument("--longest-first", choices=["auto", "off", "on"], default="auto",
                    help="scheduling of direct-method runs (ssa_set_longest_first): the library's automatic "
                         "choice (default), never, or always")
    args = ap.parse_args()
    if args.impl == "ours" and args.longest_first != "auto":
        from paper_2605_00479_gb300 import ssa
        ssa.set_longest_first(0 if args.longest_first == "off" else 2, 0)
    global N_TRAJ, MODES16
    if args.n_traj:
        N_TRAJ = args.n_traj
    if args.modes:
        MODES16 = [tuple(m.split(":")) for m in args.modes.split(",")]
    world, rank, local = dist_setup(args)
    if args.workload in ("batch", "scale"):
        if args.impl == "reference":
            run_batch_scale_reference(args, world, rank, args.workload)
        elif args.workload == "batch":
            run_batch(args, world, rank, local)
        else:
            run_scale(args, world, rank, local)
    elif args.workload in MODEL_SPECS:
        if args.impl == "reference":
            run_models_reference(args, world, rank, args.workload)
        else:
            run_models(args, world, rank, local, args.workload)
    elif args.workload != "schlogl":
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

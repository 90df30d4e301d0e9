"""Learned surrogate for the telegraph model, trained on the SSA engine's output.

Workflow (host orchestration of the CUDA kernels in libssa_gb300.so):
  1. Training data: parameter sets (kon, koff log-uniform in [0.05, 5], km in
     [5, 100], gamma in [0.5, 2]); for each, an ensemble of telegraph
     trajectories to t_end = 200 in mixed binary16 precision, run as one
     persistent batched launch; per-set histograms of the mRNA count over
     bins 0..127 (the last holding >= 127).
  2. Training: the 4 -> 256 -> 256 -> 256 -> 128 GELU network on the tensor
     cores (tcgen05 GEMMs, bf16 operands, fp32 accumulation), AdamW with a
     cosine learning-rate schedule, cross-entropy against the histograms.
  3. Serving: the network answers every query point, and the plain SSA checks
     it: each prediction is compared (Wasserstein-1, copies) with a small SSA
     ensemble of the same point (CHECK_TRAJ trajectories); a point whose
     distance exceeds the 0.5-copy threshold plus that ensemble's expected
     sampling noise (ssa_hist_w1_noise) is re-simulated with FALLBACK_TRAJ
     trajectories and answered by the SSA instead.  What the network gains is
     measured end to end against answering every point by the SSA alone
     (FALLBACK_TRAJ trajectories each), with both answers' accuracy measured
     against an independent SSA ensemble of the same size.

``python -m paper_2605_00479_gb300.surrogate`` runs the full configuration
(2^16 training sets x 1024 trajectories, 2^14 query points) and prints one
JSON line.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import presets as P
from . import ssa

BINS = 128
T_END = 200.0
LOG_LO = np.log(np.array([0.05, 0.05, 5.0, 0.5]))
LOG_HI = np.log(np.array([5.0, 5.0, 100.0, 2.0]))
W1_THRESHOLD = 0.5
CHECK_TRAJ = 64         # SSA trajectories per point that check a prediction
FALLBACK_TRAJ = 1024    # SSA trajectories per point of a re-simulated (or SSA-only) answer


def draw_parameters(n, seed):
    """[n, 4] rate tables (kon, koff, km, gamma) for the telegraph model."""
    return P.telegraph_sweep(n, seed=seed, gamma_range=(0.5, 2.0))


def standardise(params):
    """Log-parameters mapped affinely to [-1, 1] (network inputs)."""
    return (2.0 * (np.log(params) - LOG_LO) / (LOG_HI - LOG_LO) - 1.0).astype(np.float32)


def simulate_histograms(params, traj_per_set, seed, traj_offset=0, precision="mixed_f16", rounding="rn",
                        chunk_traj=2**23, stream=None):
    """Per-set mRNA histograms [n_sets, 128] (device) from SSA ensembles, in
    batched launches of at most chunk_traj trajectories (whole sets): small
    ensembles per set go in one launch, which keeps every lane busy for
    several trajectories."""
    import torch
    model = ssa.Model.from_dict(P.telegraph())
    n = params.shape[0]
    chunk_sets = max(1, chunk_traj // max(1, traj_per_set))
    out = torch.empty((n, BINS), dtype=torch.float32, device="cuda")
    for a in range(0, n, chunk_sets):
        b = min(n, a + chunk_sets)
        S = b - a
        group = {"model": model, "x0": np.tile(P.TELEGRAPH_X0, (S, 1)), "rates": params[a:b],
                 "traj_per_set": traj_per_set, "traj_offset": traj_offset + a * traj_per_set}
        batch = ssa.Batch([group], T_END, [T_END], precision, rounding, seed=seed, max_events=10**7)
        batch.launch(stream)
        counts = batch.outputs[0]["snapshots"][0, 2]
        ssa.histogram(counts, S, traj_per_set, BINS, hist=out[a:b], stream=stream)
        batch.close()
    return out


def train(net, feats, hists, steps, batch_size, lr_max=2e-3, lr_min=5e-5, weight_decay=1e-4, seed=0):
    """AdamW with a cosine schedule over minibatches of the rows shuffled once
    (then swept in order), all steps replayed on the device from one captured
    step; returns the loss trace [(step, loss)] every steps // 50 steps."""
    import torch
    n = feats.shape[0]
    g = torch.Generator(device="cuda").manual_seed(seed)
    perm = torch.randperm(n, device="cuda", generator=g)
    f, h = feats[perm].contiguous(), hists[perm].contiguous()
    every = max(1, steps // 50)
    losses = torch.full(((steps + every - 1) // every,), float("nan"), device="cuda")
    net.train(f, h, steps, batch_size, lr_max, lr_min, weight_decay, loss_every=every, loss_trace=losses)
    return [(k * every, float(v)) for k, v in enumerate(losses.cpu().tolist())]


def serve(net, query_params, seed, traj_offset, check_traj=CHECK_TRAJ, fallback_traj=FALLBACK_TRAJ):
    """Answer query points with the network, checked by the SSA.

    Returns (answers [n, 128] device, check W1 [n], fallback mask [n] device,
    number of re-simulated points)."""
    import torch
    feats = torch.from_numpy(standardise(query_params)).cuda()
    q = net.predict(feats)
    check = simulate_histograms(query_params, check_traj, seed=seed, traj_offset=traj_offset)
    w1 = ssa.hist_w1(q, check)
    noise = ssa.hist_w1_noise(q, check_traj)
    fallback = w1 > W1_THRESHOLD + noise
    idx = torch.nonzero(fallback).flatten()
    answer = q
    n_fb = int(idx.numel())
    if n_fb:
        sub = query_params[idx.cpu().numpy()]
        resim = simulate_histograms(sub, fallback_traj, seed=seed + 1, traj_offset=traj_offset)
        answer = q.clone()
        answer[idx] = resim
    return answer, w1, fallback, n_fb


def run(n_train=2**16, traj_train=1024, n_query=2**14, check_traj=CHECK_TRAJ, fallback_traj=FALLBACK_TRAJ,
        steps=6000, batch_size=1024, seed=2605):
    """The full surrogate configuration; returns a report dict."""
    import torch
    torch.cuda.synchronize()
    report = {"n_train_sets": n_train, "traj_per_set": traj_train, "n_query": n_query, "t_end": T_END,
              "bins": BINS, "precision": "mixed_f16:rn", "w1_threshold": W1_THRESHOLD}
    # 1. training data
    tr = draw_parameters(n_train, seed)
    t0 = time.perf_counter()
    h_train = simulate_histograms(tr, traj_train, seed=seed, traj_offset=0)
    torch.cuda.synchronize()
    report["data_gen_s"] = time.perf_counter() - t0
    f_train = torch.from_numpy(standardise(tr)).cuda()
    # 2. training
    net = ssa.Surrogate(max_batch=max(batch_size, n_query), seed=seed)
    t0 = time.perf_counter()
    trace = train(net, f_train, h_train, steps, batch_size, seed=seed)
    torch.cuda.synchronize()
    net.status()
    report["train_s"] = time.perf_counter() - t0
    report["train_steps"] = steps
    report["loss_first"], report["loss_last"] = trace[0][1], trace[-1][1]
    ent = -(h_train * torch.log(h_train.clamp_min(1e-30))).sum(dim=1).mean()
    report["target_entropy"] = float(ent)
    # 3. serving held-out points: the SSA alone (every point at FALLBACK_TRAJ
    # trajectories) against the network checked by small SSA ensembles; both
    # answers' accuracy against an independent SSA ensemble of each point
    qp = draw_parameters(n_query, seed + 1)
    feats_q = torch.from_numpy(standardise(qp)).cuda()
    # warm-up: one untimed pass of both paths on a few points (first uses of
    # the kernels and of the host-side selection of fallback points)
    serve(net, qp[:256], seed + 5, 2**29, check_traj, fallback_traj)
    simulate_histograms(qp[:256], fallback_traj, seed=seed + 6, traj_offset=2**29)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ssa_only = simulate_histograms(qp, fallback_traj, seed=seed + 7, traj_offset=2**31)
    torch.cuda.synchronize()
    ssa_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    answer, w1, fallback, n_fb = serve(net, qp, seed + 9, 2**30, check_traj, fallback_traj)
    torch.cuda.synchronize()
    serve_s = time.perf_counter() - t0
    twin = simulate_histograms(qp, fallback_traj, seed=seed + 8, traj_offset=2**31)   # independent reference for both
    t0 = time.perf_counter()
    reps = 20
    for _ in range(reps):
        net.predict(feats_q)
    torch.cuda.synchronize()
    nn_s = (time.perf_counter() - t0) / reps
    w1_ans = ssa.hist_w1(answer, twin).cpu().numpy()
    w1_ssa = ssa.hist_w1(ssa_only, twin).cpu().numpy()
    w1_pred = ssa.hist_w1(net.predict(feats_q), twin).cpu().numpy()
    torch.cuda.synchronize()
    report.update({
        "check_traj": check_traj, "fallback_traj": fallback_traj,
        "ssa_only_s": ssa_s, "served_s": serve_s, "speedup_end_to_end": ssa_s / serve_s,
        "surrogate_predict_s": nn_s, "speedup_predict_only": ssa_s / nn_s,
        "fallback_fraction": n_fb / n_query,
        "w1_served_vs_twin_mean": float(w1_ans.mean()), "w1_served_vs_twin_median": float(np.median(w1_ans)),
        "w1_ssa_only_vs_twin_mean": float(w1_ssa.mean()), "w1_ssa_only_vs_twin_median": float(np.median(w1_ssa)),
        "w1_prediction_vs_twin_median": float(np.median(w1_pred)),
        "served_above_1_copy": float(np.mean(w1_ans > 1.0)), "ssa_only_above_1_copy": float(np.mean(w1_ssa > 1.0)),
        "w1_check_median": float(np.median(w1.cpu().numpy())),
    })
    net.close()
    return report


if __name__ == "__main__":
    kw = {}
    for arg in sys.argv[1:]:
        k, v = arg.split("=")
        kw[k] = int(v)
    print(json.dumps(run(**kw)), flush=True)

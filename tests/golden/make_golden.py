"""Write the stored expected values under tests/golden/ (calls only oracle/).

schlogl_cme_t10.txt: law of X at t = 10 for the Schloegl model (bistable
parameter set of Sec. 4.2 in c-convention, X0 = 250, reservoirs A = 1e5 and
B = 2e5 held fixed), from the chemical master equation truncated at X <= 1500
(mass lost to the truncation < 1e-10).  Columns: x, P(X = x).

schlogl_ks_modes.json: the benchmark's accuracy criterion, computed by the
oracle.  For the benchmark's Schloegl workload (10^6-trajectory ensemble,
t_end = 10, 50 snapshots, reservoirs folded) and seeds (2605 for the reduced
modes, 2606 for an independent fp64 ensemble), the law of X at t_end of
trajectory ids 0..9999 in each mode against fp64: the two-sample KS p-value
and the Wasserstein-1 distance (scipy), and which modes pass KS p > 0.05
(the metric's criterion; the paper's Sec. 4 tables use the same test).
Usage: python make_golden.py [cme|ks|all] (default all).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cme  # noqa: E402
from paper_2605_00479_gb300 import presets  # noqa: E402


def schlogl_cme():
    m = presets.schlogl()
    x0 = presets.schlogl_x0(m)
    states, P = cme.transient(m, x0, [1500, int(x0[1]), int(x0[2])], [10.0])
    v, p = cme.marginal(states, P[0], 0)
    with open(os.path.join(HERE, "schlogl_cme_t10.txt"), "w") as f:
        f.write("# Schloegl X law at t=10 from the truncated CME (see make_golden.py)\n")
        for xv, pv in zip(v, p):
            f.write(f"{xv} {pv:.17e}\n")


KS_MODES = ["mixed_f16:rn", "mixed_bf16:rn", "uniform_f16:rn", "uniform_f16:sr", "uniform_bf16:sr",
            "uniform_f16:sra", "uniform_bf16:sra", "fp32:rn", "mixed_f16:sr", "mixed_bf16:sr"]


def schlogl_ks(n=10000, seed=2605, seed64=2606, t_end=10.0, K=50, max_events=200000):
    import json
    import oracle
    import scipy.stats as sst
    m = presets.schlogl()
    x0 = presets.schlogl_x0(m)
    samples = presets.even_samples(t_end, K)
    ref = oracle.run_parallel(m, x0, n, t_end, samples, precision="fp64", rounding="rn", normalise=True,
                              seed=seed64, max_events=max_events)["snapshots"][-1, 0].astype(np.int64)
    out = {"workload": f"schlogl bistable, X at t_end={t_end} of trajectory ids 0..{n - 1}, reservoirs folded",
           "seed": seed, "seed_fp64": seed64, "n": n, "fp64_mean": float(ref.mean()), "modes": {}}
    for key in KS_MODES:
        prec, rnd = key.split(":")
        xs = oracle.run_parallel(m, x0, n, t_end, samples, precision=prec, rounding=rnd, normalise=True, seed=seed,
                                 max_events=max_events)["snapshots"][-1, 0].astype(np.int64)
        out["modes"][key] = {"ks_p": float(sst.ks_2samp(ref, xs)[1]),
                             "w1": float(sst.wasserstein_distance(ref, xs)), "mean": float(xs.mean()),
                             "sum_x": int(xs.sum())}
        print(key, out["modes"][key], flush=True)
    out["passing"] = [k for k in KS_MODES if out["modes"][k]["ks_p"] > 0.05]
    with open(os.path.join(HERE, "schlogl_ks_modes.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("cme", "all"):
        schlogl_cme()
    if what in ("ks", "all"):
        schlogl_ks()

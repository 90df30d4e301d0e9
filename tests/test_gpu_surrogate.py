"""What the surrogate gains over the SSA alone, end to end (reduced scale of
the telegraph surrogate configuration).

Trained on SSA histograms on the tensor cores, the network answers query
points; the plain SSA checks every answer with a small ensemble (64
trajectories per point) and points whose distance exceeds the 0.5-copy
threshold plus that ensemble's expected sampling noise are re-simulated with
1024 trajectories.  Against answering every point by the SSA alone (1024
trajectories each), the served answers must come faster end to end (check,
network and re-simulation all timed), and be as accurate: both answers are
compared with an independent 1024-trajectory SSA ensemble of each point.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_surrogate_gain_over_ssa():
    from paper_2605_00479_gb300 import build
    build.build()
    from paper_2605_00479_gb300 import surrogate
    r = surrogate.run(n_train=8192, traj_train=512, n_query=4096, steps=2000, batch_size=512, seed=11)
    print(r)
    assert r["loss_last"] < r["loss_first"]
    # end to end, check + network + re-simulation against the SSA alone
    assert r["speedup_end_to_end"] > 2.0, r
    # matched accuracy against an independent ensemble of every point
    assert r["w1_served_vs_twin_mean"] <= 1.1 * r["w1_ssa_only_vs_twin_mean"], r
    assert r["served_above_1_copy"] <= r["ssa_only_above_1_copy"] + 0.02, r
    assert r["fallback_fraction"] < 0.5, r

"""What the surrogate gains over the SSA alone (reduced scale of the
telegraph surrogate configuration): trained on SSA histograms on the tensor
cores, it must answer query points much faster than simulating them, stay
within the SSA's own sampling noise of a fresh SSA ensemble for the typical
point, and send only a minority of points to the re-simulation fallback."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_surrogate_gain_over_ssa():
    from paper_2605_00479_gb300 import build
    build.build()
    from paper_2605_00479_gb300 import surrogate
    r = surrogate.run(n_train=8192, traj_train=512, n_query=2048, traj_query=512, steps=2000, batch_size=512,
                      seed=11)
    assert r["loss_last"] < r["loss_first"]
    assert r["speedup_vs_ssa"] > 100.0, r
    assert r["w1_surrogate_median"] < 1.5 * r["w1_ssa_noise_median"], r
    assert r["fallback_fraction"] < 0.5, r

"""GPU parity of the tau-leaping engine (fixed leap, every precision mode)
against the oracle, through the C ABI.

Both sides follow one contract: propensities by the direct method's rounding
chain, lambda_j = a_j tau in the mode's type, Poisson variates from the same
sampler algorithms on the same Philox words, 64-bit count updates with
clamping at zero.  Every result is integer or a binary64 leap time, so the
comparison is exact.  Step sizes are chosen so that both sampler branches
(lambda below and above 10) and clamping occur.
"""
import numpy as np
import pytest

import oracle
from paper_2605_00479_gb300 import presets as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = [("fp64", "rn"), ("fp32", "rn"), ("mixed_f16", "rn"), ("mixed_f16", "sr"), ("mixed_bf16", "rn"),
         ("mixed_bf16", "sr"), ("uniform_f16", "rn"), ("uniform_f16", "sr"), ("uniform_bf16", "rn"),
         ("uniform_bf16", "sr")]


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    assert torch.cuda.is_available()
    mod.lib()
    return mod


def general_network():
    """Species (X, Y, Z) with Z a reservoir; orders up to 3."""
    return {
        "order": np.array([[1, 0, 1], [2, 0, 0], [0, 1, 0], [0, 3, 0], [0, 0, 0], [1, 0, 0]], np.int32),
        "stoich": np.array([[1, 0, -1], [-2, 1, 0], [1, -1, 0], [0, -3, 0], [0, 1, 0], [-1, 0, 0]], np.int32),
        "rate": np.array([0.02, 0.01, 0.5, 0.001, 2.0, 0.1]),
        "law": np.zeros(6, np.int32),
        "constant": np.array([0, 0, 1], np.uint8),
    }


def pure_death():
    return {"order": np.array([[1]], np.int32), "stoich": np.array([[-1]], np.int32), "rate": np.array([1.0])}


CASES = {
    # name: (model, x0, n_traj, t_end, tau, samples, normalise)
    "birth_death_small_lambda": (P.birth_death(10.0, 0.1), [0], 1000, 100.0, 0.5, P.even_samples(100.0, 21), False),
    "birth_death_large_lambda": (P.birth_death(200.0, 1.0), [0], 777, 10.0, 0.25, P.even_samples(10.0, 11), False),
    "schlogl": (P.schlogl(), None, 96, 5.0, 0.005, P.even_samples(5.0, 26), True),
    "telegraph": (P.telegraph(0.5, 0.5, 20.0, 1.0), P.TELEGRAPH_X0, 1000, 50.0, 0.1, P.even_samples(50.0, 11), False),
    "dimer": (P.dimer(), P.dimer_x0(300), 500, 20.0, 0.05, P.even_samples(20.0, 21), False),
    "repressilator": (P.repressilator(), P.REPRESSILATOR_X0, 160, 10.0, 0.01, P.even_samples(10.0, 11), False),
    "general_network": (general_network(), [10, 5, 50], 300, 20.0, 0.1, P.even_samples(20.0, 5), True),
    "pure_death_clamped": (pure_death(), [50], 333, 20.0, 2.0, [0.0, 2.0, 4.0, 19.0, 20.0], False),
}


def gpu_tau(ssa, model_dict, x0, n_traj, t_end, tau, samples, prec, rnd, normalise, seed, state_bytes=4,
            traj_offset=0):
    m = ssa.Model.from_dict(model_dict)
    r = ssa.tau_run(m, n_traj, x0, t_end, tau, samples, prec, rnd, normalise, seed, state_bytes,
                    traj_offset=traj_offset)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in r.items()}


def assert_same(g, o):
    np.testing.assert_array_equal(g["snapshots"], o["snapshots"])
    np.testing.assert_array_equal(g["status"].view(np.uint32), o["status"])
    np.testing.assert_array_equal(g["n_events"], o["n_events"])
    np.testing.assert_array_equal(g["t_final"].view(np.uint64), o["t_final"].view(np.uint64))


def initial_state(name, model, x0):
    if x0 is None:
        return P.schlogl_x0(model)
    return x0


@pytest.mark.parametrize("prec,rnd", MODES)
@pytest.mark.parametrize("name", list(CASES))
def test_tau_parity_with_oracle(ssa, name, prec, rnd):
    model, x0, n, t_end, tau, samples, norm = CASES[name]
    x0 = initial_state(name, model, x0)
    seed = 1000 + len(name)
    g = gpu_tau(ssa, model, x0, n, t_end, tau, samples, prec, rnd, norm, seed)
    o = oracle.tau_run(model, x0, n, t_end, tau, samples, precision=prec, rounding=rnd, normalise=norm, seed=seed)
    assert_same(g, o)
    if name == "pure_death_clamped":
        assert np.any(o["status"] & 16)


def test_tau_both_sampler_branches_and_clamping_occur():
    """The cases above reach lambda >= 10 (transformed rejection) and clamping."""
    model, x0, n, t_end, tau, samples, norm = CASES["birth_death_large_lambda"]
    o = oracle.tau_run(model, x0, 50, t_end, tau, samples, precision="fp32", seed=1)
    assert o["snapshots"][-1, 0].mean() > 40 * 4        # death lambda = x tau >> 10 at stationarity
    model, x0, n, t_end, tau, samples, norm = CASES["telegraph"]
    o = oracle.tau_run(model, x0, n, t_end, tau, samples, precision="fp64", seed=1)
    assert np.any(o["status"] & 16)


@pytest.mark.parametrize("prec,rnd", [("fp32", "rn"), ("uniform_bf16", "sr")])
def test_tau_overflow_and_nan(ssa, prec, rnd):
    big = {"order": np.array([[0]], np.int32), "stoich": np.array([[1]], np.int32), "rate": np.array([3e38])}
    g = gpu_tau(ssa, big, [7], 70, 10.0, 10.0, [10.0], prec, rnd, False, 1)
    o = oracle.tau_run(big, [7], 70, 10.0, 10.0, [10.0], precision=prec, rounding=rnd, seed=1)
    assert_same(g, o)
    assert np.all(o["status"] & 1)
    hill = P.hill_self(alpha0=1.0, alpha=1e6, h=2, gamma=1.0)
    g = gpu_tau(ssa, hill, [300], 70, 1.0, 0.5, [0.5, 1.0], "uniform_f16", "sr", False, 2)
    o = oracle.tau_run(hill, [300], 70, 1.0, 0.5, [0.5, 1.0], precision="uniform_f16", rounding="sr", seed=2)
    assert_same(g, o)
    assert np.all(o["status"] & 8)


def test_tau_ragged_offset_int16_and_launch_shape(ssa):
    """Ragged ensemble, trajectory ids near 2^32, int16 snapshots and several
    launch shapes all give the oracle's results."""
    model = P.dimer()
    x0 = P.dimer_x0(300)
    n, off = 1037, 2**32 - 1037
    samples = P.even_samples(5.0, 6)
    o = oracle.tau_run(model, x0, n, 5.0, 0.05, samples, precision="mixed_bf16", rounding="sr", seed=77,
                       state_bytes=2, g0=off)
    try:
        for block, per_sm in [(128, 0), (32, 1), (256, 2)]:
            ssa.set_launch_config(block, per_sm, 1)
            g = gpu_tau(ssa, model, x0, n, 5.0, 0.05, samples, "mixed_bf16", "sr", False, 77, state_bytes=2,
                        traj_offset=off)
            assert g["snapshots"].dtype == np.int16
            assert_same(g, o)
    finally:
        ssa.set_launch_config()


def test_tau_single_leap_and_off_grid_end(ssa):
    """t_end below tau (one leap) and t_end off the leap grid (ceil)."""
    model = P.birth_death(10.0, 0.1)
    for t_end, tau in [(0.3, 1.0), (1.0, 0.3)]:
        samples = [0.0, t_end]
        g = gpu_tau(ssa, model, [5], 200, t_end, tau, samples, "uniform_f16", "rn", False, 4)
        o = oracle.tau_run(model, [5], 200, t_end, tau, samples, precision="uniform_f16", rounding="rn", seed=4)
        assert_same(g, o)
        assert np.all(o["t_final"] == np.ceil(t_end / tau) * tau)


def test_tau_outputs_in_page_locked_host_memory(ssa):
    """Page-locked host buffers passed as the outputs: the kernel writes into
    host memory directly; results equal the device-buffer run."""
    md = P.schlogl()
    x0 = P.schlogl_x0(md)
    m = ssa.Model.from_dict(md)
    n, samples = 50001, P.even_samples(2.0, 5)
    host = {"out": torch.full((5, m.N, n), -9, dtype=torch.int32).pin_memory(),
            "status": torch.full((n,), -9, dtype=torch.int32).pin_memory(),
            "n_events": torch.full((n,), -9, dtype=torch.int64).pin_memory(),
            "t_final": torch.full((n,), -9.0, dtype=torch.float64).pin_memory()}
    ssa.tau_run(m, n, x0, 2.0, 0.005, samples, "uniform_bf16", "sr", True, 21, traj_offset=99, **host)
    torch.cuda.synchronize()
    g = gpu_tau(ssa, md, x0, n, 2.0, 0.005, samples, "uniform_bf16", "sr", True, 21, traj_offset=99)
    np.testing.assert_array_equal(host["out"].numpy(), g["snapshots"])
    np.testing.assert_array_equal(host["status"].numpy(), g["status"])
    np.testing.assert_array_equal(host["n_events"].numpy(), g["n_events"])
    np.testing.assert_array_equal(host["t_final"].numpy().view(np.uint64), g["t_final"].view(np.uint64))

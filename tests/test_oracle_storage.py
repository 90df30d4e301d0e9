"""int16 snapshot storage is an output format: it never changes a trajectory.
A run with int16 storage equals the int32 run with every snapshot clamped to
[-32768, 32767]; the STATE_RANGE bit (4) is added exactly where a stored value
was clamped; event counts and final times are identical.  Only a negative
count (the Sec. 2 update leaving the state space) ends a trajectory."""
import numpy as np
import pytest

import oracle
from paper_2605_00479_gb300 import presets as P


def _check_storage(a, b, axis_traj):
    s32, s16 = a["snapshots"].astype(np.int64), b["snapshots"].astype(np.int64)
    np.testing.assert_array_equal(s16, np.clip(s32, -32768, 32767))
    clamped = np.any((s32 > 32767) | (s32 < -32768), axis=tuple(i for i in range(s32.ndim) if i != axis_traj))
    np.testing.assert_array_equal(b["status"], a["status"] | np.where(clamped, 4, 0).astype(np.uint32))
    np.testing.assert_array_equal(a["n_events"], b["n_events"])
    np.testing.assert_array_equal(a["t_final"].view(np.uint64), b["t_final"].view(np.uint64))
    return clamped


@pytest.mark.parametrize("prec,rnd", [("fp64", "rn"), ("fp32", "rn"), ("mixed_f16", "sr"), ("uniform_bf16", "sr")])
def test_direct_method_int16_storage_is_output_only(prec, rnd):
    md = P.schlogl()                     # reservoirs A = 1e5, B = 2e5 do not fit int16
    x0 = P.schlogl_x0(md)
    kw = dict(precision=prec, rounding=rnd, normalise=True, seed=3, max_events=10**6)
    a = oracle.run(md, x0, 40, 1.0, P.even_samples(1.0, 4), state_bytes=4, **kw)
    b = oracle.run(md, x0, 40, 1.0, P.even_samples(1.0, 4), state_bytes=2, **kw)
    clamped = _check_storage(a, b, 2)
    assert clamped.all() and a["n_events"].min() > 100


def test_negative_count_still_ends_the_trajectory():
    neg = {"order": np.array([[0]]), "stoich": np.array([[-1]]), "rate": np.array([1.0]), "law": np.array([0])}
    for sb in (2, 4):
        r = oracle.run(neg, [2], 20, 100.0, [100.0], "fp64", "rn", False, 5, 10**6, state_bytes=sb)
        assert np.all(r["status"] == 4) and np.all(r["n_events"] == 3) and np.all(r["snapshots"] == -1)


def test_rdme_int16_storage_is_output_only():
    m = P.birth_death(4000.0, 0.0)       # pure birth: counts pass 32767 inside the run
    x0 = np.zeros((2, 1), np.int32)
    kw = dict(precision="fp32", rounding="rn", seed=4, max_events=10**6)
    a = oracle.rdme_run(m, (2,), [1.0], x0, 6, 10.0, [5.0, 10.0], state_bytes=4, **kw)
    b = oracle.rdme_run(m, (2,), [1.0], x0, 6, 10.0, [5.0, 10.0], state_bytes=2, **kw)
    clamped = _check_storage(a, b, 3)
    assert clamped.all()
    assert a["snapshots"][0].min() > 10000 and a["snapshots"][1].min() > 32767


def test_species_mask_stores_a_subset_and_clamps_only_stored_species():
    """out_species: the snapshots hold the chosen species in ascending order,
    identical to the full output's rows; the trajectories are unchanged; the
    int16 clamp flag comes only from stored species (the Schloegl reservoirs
    A = 1e5, B = 2e5 clamp when stored, not when left out)."""
    m = P.schlogl()
    x0 = P.schlogl_x0(m)
    smp = P.even_samples(1.0, 4)
    full = oracle.run(m, x0, 40, 1.0, smp, "mixed_f16", "sr", True, 3, 10**6, state_bytes=2)
    only_x = oracle.run(m, x0, 40, 1.0, smp, "mixed_f16", "sr", True, 3, 10**6, state_bytes=2, out_species=0b001)
    assert only_x["snapshots"].shape == (4, 1, 40)
    np.testing.assert_array_equal(only_x["snapshots"][:, 0], full["snapshots"][:, 0])
    np.testing.assert_array_equal(only_x["n_events"], full["n_events"])
    np.testing.assert_array_equal(only_x["t_final"], full["t_final"])
    assert np.all(full["status"] & oracle.STATUS_STATE_RANGE)
    assert not np.any(only_x["status"] & oracle.STATUS_STATE_RANGE)
    xb = oracle.run(m, x0, 40, 1.0, smp, "mixed_f16", "sr", True, 3, 10**6, state_bytes=4, out_species=0b101)
    full4 = oracle.run(m, x0, 40, 1.0, smp, "mixed_f16", "sr", True, 3, 10**6, state_bytes=4)
    np.testing.assert_array_equal(xb["snapshots"], full4["snapshots"][:, [0, 2]])
    import pytest
    with pytest.raises(ValueError):
        oracle.run(m, x0, 4, 1.0, smp, "fp64", "rn", True, 3, 10**6, out_species=0b1000)

"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every function include/ssa.h declares, and rejects invalid arguments
on the host before anything is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2605_00479_gb300 import presets as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ssa():
    from paper_2605_00479_gb300 import build, ssa as mod
    build.build()
    return mod


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ssa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssa_\w+)\s*\(", text)))


def test_library_exports_every_declared_function(ssa):
    names = declared_functions()
    assert len(names) >= 7
    L = ctypes.CDLL(ssa.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
        assert n in ssa.SIGNATURES, n


def test_structure_families(ssa):
    assert ssa.Model.from_dict(P.birth_death()).family == "birth_death"
    assert ssa.Model.from_dict(P.schlogl()).family == "schlogl"
    assert ssa.Model.from_dict(P.telegraph()).family == "telegraph"
    assert ssa.Model.from_dict(P.dimer()).family == "dimer"
    assert ssa.Model.from_dict(P.repressilator()).family == "repressilator"
    assert ssa.Model.from_dict(P.repressilator(h=3)).family == "general"
    assert ssa.Model.from_dict(P.hill_self()).family == "general"


@pytest.mark.parametrize("bad", ["order", "N", "M", "hill_h", "hill_reg", "rate_nan", "rate_neg", "law"])
def test_model_create_rejects(ssa, bad):
    m = {k: (None if v is None else np.array(v, copy=True)) for k, v in P.repressilator().items() if k != "names"}
    order, stoich = m["order"], m["stoich"]
    if bad == "order":
        order[1, 0] = 4
    elif bad == "N":
        order, stoich = np.zeros((2, 9), np.int32), np.zeros((2, 9), np.int32)
        m["rate"], m["law"], m["hill"] = np.ones(2), None, None
    elif bad == "M":
        order, stoich = np.zeros((17, 1), np.int32), np.zeros((17, 1), np.int32)
        m["rate"], m["law"], m["hill"] = np.ones(17), None, None
    elif bad == "hill_h":
        m["hill"][0, 2] = 0
    elif bad == "hill_reg":
        m["hill"][0, 3] = 6
    elif bad == "rate_nan":
        m["rate"][1] = np.nan
    elif bad == "rate_neg":
        m["rate"][1] = -1.0
    elif bad == "law":
        m["law"][1] = 7
    with pytest.raises(ssa.SSAError) as e:
        ssa.Model(order, stoich, m["rate"], m["law"], m["hill"])
    assert e.value.code == ssa.SSA_EINVAL


@pytest.mark.parametrize("case", ["precision", "sr_fp64", "sra_mixed", "t_end", "unsorted", "beyond", "no_samples", "state_bytes",
                                  "max_events", "ids", "x0"])
def test_run_rejects_before_launch(ssa, case):
    m = ssa.Model.from_dict(P.birth_death())
    kw = dict(n_traj=4, x0=[0], t_end=10.0, sample_times=[0.0, 5.0, 10.0], precision="fp32", rounding="rn",
              seed=0, max_events=100, state_bytes=4, traj_offset=0)
    if case == "precision":
        kw["precision"] = 9
    elif case == "sr_fp64":
        kw["precision"], kw["rounding"] = "fp64", "sr"
    elif case == "sra_mixed":
        kw["precision"], kw["rounding"] = "mixed_f16", "sra"
    elif case == "t_end":
        kw["t_end"] = 0.0
    elif case == "unsorted":
        kw["sample_times"] = [5.0, 1.0]
    elif case == "beyond":
        kw["sample_times"] = [11.0]
    elif case == "no_samples":
        kw["sample_times"] = []
    elif case == "state_bytes":
        kw["state_bytes"] = 3
    elif case == "max_events":
        kw["max_events"] = -1
    elif case == "ids":
        kw["traj_offset"] = 2**32 - 2
    elif case == "x0":
        kw["x0"] = [-1]
    out = np.zeros(12, np.int32)
    st = np.zeros(4, np.uint32)
    with pytest.raises(ssa.SSAError) as e:
        ssa.ensemble_run_host(m, out=out.reshape(-1, 1, 4)[:max(1, len(kw["sample_times"]))] if kw["sample_times"] else None,
                              status=st, **kw)
    assert e.value.code == ssa.SSA_EINVAL


def test_launch_config_validation(ssa):
    with pytest.raises(ssa.SSAError):
        ssa.set_launch_config(48, 0, 1)
    with pytest.raises(ssa.SSAError):
        ssa.set_launch_config(512, 0, 1)
    ssa.set_launch_config()


def test_tail_compaction_switch_validation(ssa):
    assert ssa.lib().ssa_set_tail_compaction(2) == ssa.SSA_EINVAL
    assert ssa.lib().ssa_set_tail_compaction(-1) == ssa.SSA_EINVAL
    ssa.set_tail_compaction(False)
    ssa.set_tail_compaction(True)


def test_longest_first_switch_validation(ssa):
    L = ssa.lib()
    assert L.ssa_set_longest_first(3, 0) == ssa.SSA_EINVAL
    assert L.ssa_set_longest_first(-1, 0) == ssa.SSA_EINVAL
    assert L.ssa_set_longest_first(2, 1) == ssa.SSA_EINVAL      # odd: would park inside a step pair
    assert L.ssa_set_longest_first(2, 4097) == ssa.SSA_EINVAL
    assert L.ssa_set_longest_first(2, -2) == ssa.SSA_EINVAL
    ssa.set_longest_first(2, 2)
    ssa.set_longest_first(0, 0)
    ssa.set_longest_first()
    assert L.ssa_direct_kernel_launches(None) == ssa.SSA_EINVAL
    assert ssa.direct_kernel_launches() >= 0


def test_batch_create_rejects_before_allocating(ssa):
    """Group validation happens on the host before any device allocation."""
    m = ssa.Model.from_dict(P.telegraph())
    x0 = np.ascontiguousarray(np.tile(P.TELEGRAPH_X0, (2, 1)), dtype=np.int32)
    bad_rates = np.array([[0.1, 0.1, 5.0, 1.0], [0.1, -1.0, 5.0, 1.0]])
    samples = np.array([10.0])
    L = ssa.lib()
    for rates, n_groups in [(bad_rates, 1), (None, 0), (None, 17)]:
        arr = (ssa.BatchGroup * 1)()
        arr[0] = ssa.BatchGroup(m.handle, 2, 4, ssa._np_ptr(rates), None, ssa._np_ptr(x0), 0, None, None, None, None)
        h = ctypes.c_void_p()
        rc = L.ssa_batch_create(n_groups, ctypes.cast(arr, ctypes.c_void_p), 10.0, 1, ssa._np_ptr(samples), 2, 0, 0,
                                0, 1000, 4, ctypes.byref(h))
        assert rc == ssa.SSA_EINVAL and not h.value
    # outputs missing for a non-empty group
    arr = (ssa.BatchGroup * 1)()
    arr[0] = ssa.BatchGroup(m.handle, 2, 4, None, None, ssa._np_ptr(x0), 0, None, None, None, None)
    h = ctypes.c_void_p()
    assert L.ssa_batch_create(1, ctypes.cast(arr, ctypes.c_void_p), 10.0, 1, ssa._np_ptr(samples), 2, 0, 0, 0, 1000,
                              4, ctypes.byref(h)) == ssa.SSA_EINVAL


@pytest.mark.parametrize("case", ["tau_zero", "tau_nan", "too_many_leaps", "sra", "sr_fp64", "t_end", "state_bytes"])
def test_tau_run_rejects_before_launch(ssa, case):
    """ssa_tau_run validates on the host (no device pointer is touched)."""
    m = ssa.Model.from_dict(P.birth_death())
    x0 = np.zeros(1, np.int32)
    st = np.array([0.0, 5.0, 10.0])
    t_end, tau, prec, rnd, sb = 10.0, 0.1, ssa.PRECISION["fp32"], 0, 4
    if case == "tau_zero":
        tau = 0.0
    elif case == "tau_nan":
        tau = float("nan")
    elif case == "too_many_leaps":
        tau = 1e-9
    elif case == "sra":
        prec, rnd = ssa.PRECISION["uniform_f16"], ssa.ROUNDING["sra"]
    elif case == "sr_fp64":
        prec, rnd = ssa.PRECISION["fp64"], ssa.ROUNDING["sr"]
    elif case == "t_end":
        t_end = float("inf")
    elif case == "state_bytes":
        sb = 8
    fake = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    rc = ssa.lib().ssa_tau_run(m.handle, 4, 0, x0.ctypes.data, t_end, tau, 3, st.ctypes.data, prec, rnd, 0, 0, sb,
                               fake, fake, None, None, None)
    assert rc == ssa.SSA_EINVAL
    assert ssa.lib().ssa_last_error()


def test_tau_run_empty_ensemble_is_a_no_op(ssa):
    m = ssa.Model.from_dict(P.birth_death())
    x0 = np.zeros(1, np.int32)
    st = np.array([10.0])
    rc = ssa.lib().ssa_tau_run(m.handle, 0, 0, x0.ctypes.data, 10.0, 0.5, 1, st.ctypes.data, 0, 0, 0, 0, 4,
                               None, None, None, None, None)
    assert rc == ssa.SSA_OK


@pytest.mark.parametrize("case", ["dims", "too_many_voxels", "no_fit", "neg_diffusion", "constant_diffuses",
                                  "constant_uneven", "sra", "max_events", "neg_x0"])
def test_rdme_run_rejects_before_launch(ssa, case):
    """ssa_rdme_run validates on the host before any device call."""
    m = ssa.Model.from_dict(P.dimer())
    nx, ny, nz = 4, 2, 1
    D = np.array([1.0, 0.5])
    prec, rnd, cap = ssa.PRECISION["fp32"], 0, 1000
    if case in ("constant_diffuses", "constant_uneven"):
        m = ssa.Model.from_dict(P.schlogl())
        D = np.array([1.0, 0.0, 0.0])
    S = nx * ny * nz
    x0 = np.ones((S, m.N), np.int32) * 5
    if case == "dims":
        nz = 0
    elif case == "too_many_voxels":
        nx, ny, nz = 64, 32, 1
    elif case == "no_fit":
        nx, ny, nz, prec = 32, 32, 1, ssa.PRECISION["fp64"]
        x0 = np.ones((1024, m.N), np.int32)
    elif case == "neg_diffusion":
        D[0] = -1.0
    elif case == "constant_diffuses":
        D[1] = 0.5
    elif case == "constant_uneven":
        x0[3, 2] += 1
    elif case == "sra":
        prec, rnd = ssa.PRECISION["uniform_f16"], ssa.ROUNDING["sra"]
    elif case == "max_events":
        cap = 2**32
    elif case == "neg_x0":
        x0[5, 1] = -1
    st = np.array([0.0, 1.0])
    fake = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    rc = ssa.lib().ssa_rdme_run(m.handle, nx, ny, nz, D.ctypes.data, 4, 0, x0.ctypes.data, 1.0, 2, st.ctypes.data,
                                prec, rnd, 0, 0, cap, 4, fake, fake, None, None, None)
    assert rc == ssa.SSA_EINVAL, case
    assert ssa.lib().ssa_last_error()


def test_rdme_run_empty_ensemble_is_a_no_op(ssa):
    m = ssa.Model.from_dict(P.dimer())
    x0 = np.ones((3, 2), np.int32)
    D = np.array([1.0, 1.0])
    st = np.array([1.0])
    rc = ssa.lib().ssa_rdme_run(m.handle, 3, 1, 1, D.ctypes.data, 0, 0, x0.ctypes.data, 1.0, 1, st.ctypes.data,
                                0, 0, 0, 0, 100, 4, None, None, None, None, None)
    assert rc == ssa.SSA_OK


def test_statistics_entry_points_reject_before_launch(ssa):
    """Argument checks of the ensemble-statistics entry points (no device use)."""
    L = ssa.lib()
    fake = ctypes.c_void_p(16)
    assert L.ssa_count_histogram(fake, 3, 10, 8, fake, fake, None) == ssa.SSA_EINVAL      # element size
    assert L.ssa_count_histogram(fake, 4, 10, 0, fake, fake, None) == ssa.SSA_EINVAL      # bins
    assert L.ssa_count_histogram(None, 4, 10, 8, fake, fake, None) == ssa.SSA_EINVAL     # values
    assert L.ssa_count_histogram(None, 4, 0, 8, None, None, None) == ssa.SSA_OK          # empty
    assert L.ssa_hist_ks_w1(None, fake, 8, fake, None) == ssa.SSA_EINVAL
    assert L.ssa_hist_ks_w1(fake, fake, 1 << 25, fake, None) == ssa.SSA_EINVAL
    assert L.ssa_dwell_histogram(fake, 4, 10, 100, 50, fake, None) == ssa.SSA_EINVAL      # k_stride < n
    assert L.ssa_dwell_histogram(fake, 4, 0, 100, 100, fake, None) == ssa.SSA_EINVAL      # K
    assert L.ssa_dwell_histogram(None, 4, 10, 0, 0, None, None) == ssa.SSA_OK

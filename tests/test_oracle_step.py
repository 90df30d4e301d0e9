"""Independent pin of the oracle's reduced-precision direct-method step.

The oracle (oracle/ssa_oracle.c) computes the 16-bit modes with integer
operations on bit patterns.  Here one step is recomputed from the paper's
definitions alone, in plain Python/numpy, and compared element by element
with what the oracle recorded while it ran (oracle.trace_step):

* the paper's Sec. 2 direct-method step: propensities, partial sums S_j,
  a0 = S_M, tau = -ln(u1)/a0, the smallest mu with S_mu > u2 a0, t + tau;
* the mode partition of Sec. 3.2 / Sec. 4: mixed modes round only the
  propensity chain to 16 bits (sums, time and variates in binary32), uniform
  modes round every operation (reading R7 for the variates);
* one 16-bit operation = the binary32 operation on the widened operands, then
  one rounding (reading R4).  Round to nearest is numpy's float16 conversion
  and torch's bfloat16 conversion (library routines).  Stochastic rounding is
  written from the values, Sec. 3.3: with x- <= |x| < x+ the neighbouring
  16-bit values and frac = (|x| - x-)/(x+ - x-), the result is x+ exactly
  when r + frac 2^R >= 2^R for the operation's R-bit random value r (R = 13
  for binary16, 16 for bfloat16, reading R5); beyond the largest finite value
  it is infinity;
* random numbers from the published Philox4x32-10 (pinned by its known-answer
  vectors elsewhere) on the schedule of reading R6, and ln from the oracle's
  own logarithm (pinned to 2 ulp elsewhere).

States are chosen where the chains really round: Schloegl X = 300, 560 and
2100 (bf16 is exact only to 256, binary16 to 2048), the dimer at 300
monomers, repressilator Hill terms at repressor counts 5, 300 and 2000, and
steps deep inside trajectories (t > 0, Philox blocks beyond the first).
A dropped term, a swapped operand order, a wrong SR slot or random half, or
a mis-rounded variate changes at least one compared value.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2605_00479_gb300 import presets as P

F32 = np.float32


# ------------------------------------------------------------ roundings
def rn16(x, fmt):
    """Round-to-nearest-even of a binary32 value to the 16-bit type (library)."""
    x = F32(x)
    if fmt == "f16":
        with np.errstate(over="ignore"):
            return float(np.float16(x))
    return float(torch.tensor(float(x), dtype=torch.float32).to(torch.bfloat16).item())


def _quantum(ax, fmt):
    """Spacing of the 16-bit type at |x| (definition of the formats:
    binary16 1/5/10 bits, emin -14; bfloat16 1/8/7 bits, emin -126)."""
    e = math.frexp(ax)[1] - 1 if ax > 0 else -1000
    if fmt == "f16":
        return 2.0 ** (max(e, -14) - 10)
    return 2.0 ** (max(e, -126) - 7)


def sr16(x, r16, fmt):
    """Stochastic rounding of a binary32 value with a 16-bit random value."""
    x = float(F32(x))
    if x == 0.0 or not math.isfinite(x):
        return x
    ax = abs(x)
    q = _quantum(ax, fmt)
    lo = math.floor(ax / q) * q
    if lo == ax:
        return x
    R = 13 if fmt == "f16" else 16
    frac = (ax - lo) / q
    r = r16 & ((1 << R) - 1)
    y = lo + q if r + frac * 2.0**R >= 2.0**R else lo
    top = 65504.0 if fmt == "f16" else float(np.finfo(np.float32).max)
    if y > top:
        y = math.inf
    return math.copysign(y, x)


# ------------------------------------------------------------ random words
def philox_word(seed, g, stream, w):
    """Word w of a trajectory's Philox stream (block w // 4, lane w % 4)."""
    blk = w // 4
    out = oracle.philox([blk & 0xFFFFFFFF, blk >> 32, g, stream], [seed & 0xFFFFFFFF, seed >> 32])
    return int(out[0][w % 4])


# ------------------------------------------------------------ one step
def chain_ops(model, j, folded):
    law = int(model.get("law", np.zeros(len(model["rate"])))[j])
    if law == 1:
        return int(model["hill"][j][2]) + 3
    return int(sum(2 * model["order"][j][i] for i in range(len(model["order"][j])) if not folded[i]))


def rate_constants(model, x0, normalise):
    """R1: c'_j = c_j / prod r! (binary64), reservoir counts folded in when
    normalising (the paper's k1 A, k3 B of the rescaled Schloegl set)."""
    order = np.asarray(model["order"])
    M, N = order.shape
    const = np.asarray(model.get("constant", np.zeros(N)), dtype=bool)
    cp, folded = [], []
    for j in range(M):
        c = float(model["rate"][j])
        for i in range(N):
            c = c / math.factorial(int(order[j][i]))
        fj = [bool(normalise and const[i] and order[j][i] > 0) for i in range(N)]
        for i in range(N):
            if fj[i]:
                for m in range(int(order[j][i])):
                    c = c * float(x0[i] - m)
        cp.append(c)
        folded.append(fj)
    return cp, folded


def recompute_step(model, x0, x, t, n, g, seed, prec, rounding, normalise, plant=None):
    """One step from the definitions.  ``plant`` injects a plausible mistake
    (for the test that the comparison can see it): 'half' swaps the halves
    of the SR words, 'factor_order' multiplies a chain's factors in reverse,
    'sum_slot' shifts the partial sums' SR slots by one, 'target_u2' forms
    the target from the unrounded u2."""
    order = np.asarray(model["order"])
    M, N = order.shape
    law = np.asarray(model.get("law", np.zeros(M)), dtype=int)
    hill = np.asarray(model["hill"]).reshape(M, 4) if model.get("hill") is not None else None
    fmt = "bf16" if prec.endswith("bf16") else "f16"
    mixed, uniform = prec.startswith("mixed"), prec.startswith("uniform")
    sr_chain = rounding == "sr"
    sr_acc = rounding in ("sr", "sra") and uniform
    cp, folded = rate_constants(model, x0, normalise)
    # number of SR operations per step, and this step's first SR word
    nsr = sum(chain_ops(model, j, folded[j]) for j in range(M))
    if uniform:
        nsr += (M - 1) + 5
    if rounding == "sra":
        nsr = M
    blocks = (nsr + 7) // 8
    base_word = 4 * n * blocks

    def rbits(op):
        w = philox_word(seed, g, 1, base_word + op // 2)
        odd = bool(op & 1) != (plant == "half")
        return (w >> 16) if odd else (w & 0xFFFF)

    def rnd(v, op, stochastic):
        return sr16(v, rbits(op), fmt) if stochastic else rn16(v, fmt)

    if prec == "fp64":
        conv = float
    elif prec == "fp32":
        conv = lambda v: float(F32(v))   # noqa: E731
    else:
        conv = lambda v: rn16(float(F32(v)), fmt)   # noqa: E731  (c' once, by RN)
    c16 = [conv(c) for c in cp]
    a = []
    op = 0
    for j in range(M):
        start = op
        if prec in ("fp64", "fp32"):
            T = float if prec == "fp64" else F32
            if law[j] == 1:
                h, reg = int(hill[j][2]), int(hill[j][3])
                Pv = T(x[reg])
                qv = Pv
                for _ in range(h - 1):
                    qv = T(qv * Pv)
                dv = T(T(1.0) + qv)
                fv = T(T(conv(hill[j][1])) / dv)
                a.append(float(T(T(conv(hill[j][0])) + fv)))
            elif any(order[j][i] > 0 and not folded[j][i] and x[i] < order[j][i] for i in range(N)):
                a.append(0.0)
            else:
                v = T(c16[j])
                for i in range(N):
                    if folded[j][i]:
                        continue
                    for m in range(int(order[j][i])):
                        v = T(v * T(x[i] - m))
                a.append(float(v))
            continue
        if law[j] == 1:
            h, reg = int(hill[j][2]), int(hill[j][3])
            a0h, a1h = conv(hill[j][0]), conv(hill[j][1])
            Pv = rnd(F32(x[reg]), op, sr_chain)
            op += 1
            qv = Pv
            for _ in range(h - 1):
                qv = rnd(F32(qv) * F32(Pv), op, sr_chain)
                op += 1
            dv = rnd(F32(1.0) + F32(qv), op, sr_chain)
            fv = rnd(F32(a1h) / F32(dv), op + 1, sr_chain)
            a.append(rnd(F32(a0h) + F32(fv), op + 2, sr_chain))
        elif any(order[j][i] > 0 and not folded[j][i] and x[i] < order[j][i] for i in range(N)):
            a.append(0.0)
        else:
            v = c16[j]
            for i in range(N):
                if folded[j][i]:
                    continue
                ms = range(int(order[j][i]))
                for m in (reversed(ms) if plant == "factor_order" else ms):
                    f = rnd(F32(x[i] - m), op, sr_chain)
                    v = rnd(F32(v) * F32(f), op + 1, sr_chain)
                    op += 2
            a.append(v)
        op = start + chain_ops(model, j, folded[j])
    # partial sums
    S = [a[0]]
    for j in range(1, M):
        if prec == "fp64":
            S.append(S[-1] + a[j])
        elif uniform:
            slot = (j - 1) if rounding == "sra" else op + (j - 1) + (plant == "sum_slot")
            S.append(rnd(F32(S[-1]) + F32(a[j]), slot, sr_acc))
        else:
            S.append(float(F32(S[-1]) + F32(a[j])))
    a0 = S[-1]
    w0 = philox_word(seed, g, 0, 2 * n)
    w1 = philox_word(seed, g, 0, 2 * n + 1)
    if prec == "fp64":
        u1 = (w0 + 1.0) * 2.0**-32
        u2 = w1 * 2.0**-32
        E = -float(oracle.log_f64(np.array([u1]))[0])
        U2, tau, target = u2, E / a0, u2 * a0
        t_new = t + tau
    else:
        u1 = float(F32(((w0 >> 8) + 1) * 2.0**-24))
        u2 = float(F32((w1 >> 8) * 2.0**-24))
        lg = float(-oracle.log_f32(np.array([u1], np.float32))[0])
        if uniform:
            v0 = op + (M - 1)
            E = rnd(lg, v0, sr_chain)
            U2 = rnd(u2, v0 + 1, sr_chain)
            tau = rnd(F32(E) / F32(a0), v0 + 2, sr_chain)
            target = rnd(F32(u2 if plant == "target_u2" else U2) * F32(a0), v0 + 3, sr_chain)
            t_new = rnd(F32(t) + F32(tau), (M - 1) if rounding == "sra" else v0 + 4, sr_acc)
        else:
            E, U2 = lg, u2
            tau = float(F32(E) / F32(a0))
            target = float(F32(u2) * F32(a0))
            t_new = float(F32(t) + F32(tau))
    mu = next((j for j in range(M) if S[j] > target), None)
    if mu is None:
        mu = max((j for j in range(M) if a[j] > 0), default=-1)
    return {"a": np.array(a), "S": np.array(S), "a0": a0, "u1": u1, "u2": u2, "E": E, "U2": U2, "tau": tau,
            "target": target, "t_new": t_new, "mu": mu}


def check(model, x0, step, prec, rounding, normalise, seed, g):
    tr = oracle.trace_step(model, x0, step, prec, rounding, normalise, seed=seed, g=g)
    if tr is None and step == 0:
        # the first step did not run to the selection: the recomputed a0 must
        # be infinite (binary16 overflow, the paper's OVF rows) and the oracle
        # must have stopped with OVERFLOW before any event
        mine = recompute_step(model, x0, np.asarray(x0), 0.0, 0, g, seed, prec, rounding, normalise)
        assert math.isinf(mine["a0"]), mine["a0"]
        o = oracle.run(model, x0, 1, 1e30, [1e30], prec, rounding, normalise, seed, max_events=1, g0=g)
        assert o["status"][0] & oracle.STATUS_OVERFLOW and o["n_events"][0] == 0
        return None
    assert tr is not None, "the trajectory ended before the traced step"
    mine = recompute_step(model, x0, tr["x"], tr["t"], tr["n"], g, seed, prec, rounding, normalise)
    for key in ("a", "S"):
        np.testing.assert_array_equal(np.asarray(tr[key]), mine[key], err_msg=key)
    for key in ("a0", "u1", "u2", "E", "U2", "tau", "target", "t_new", "mu"):
        got, exp = tr[key], mine[key]
        assert got == exp or (math.isnan(got) and math.isnan(exp)), (key, got, exp, prec, rounding)
    return tr


MODES = [(p, r) for p in ("mixed_f16", "mixed_bf16", "uniform_f16", "uniform_bf16") for r in ("rn", "sr")]
MODES += [("uniform_f16", "sra"), ("uniform_bf16", "sra"), ("fp32", "rn"), ("fp64", "rn")]


def _schlogl_at(X):
    m = P.schlogl()
    x0 = np.array(P.schlogl_x0(m), dtype=np.int32)
    x0[0] = X
    return m, x0


@pytest.mark.parametrize("prec,rounding", MODES)
@pytest.mark.parametrize("X", [300, 560, 2100])
def test_schlogl_step_where_chains_round(prec, rounding, X):
    m, x0 = _schlogl_at(X)
    for g in (0, 7, 123456):
        check(m, x0, 0, prec, rounding, True, seed=11 + X, g=g)


@pytest.mark.parametrize("prec,rounding", MODES)
def test_dimer_and_repressilator_steps(prec, rounding):
    d = P.dimer()
    check(d, P.dimer_x0(300), 0, prec, rounding, False, seed=5, g=3)
    r = P.repressilator()
    for pv in (5, 300, 2000):
        x0 = np.array(P.REPRESSILATOR_X0, dtype=np.int32)
        x0[3:] = [pv, pv // 2 + 1, 2 * pv]        # repressors (proteins) at different levels
        x0[:3] = [10, 0, 37]
        check(r, x0, 0, prec, rounding, False, seed=9 + pv, g=pv)


@pytest.mark.parametrize("prec,rounding", MODES)
def test_steps_deep_inside_trajectories(prec, rounding):
    """Later steps: t > 0 enters the clock update, the Philox counter runs
    past its first blocks, and the SR words come from step n's blocks."""
    m, x0 = _schlogl_at(250)
    for step in (1, 40, 1001):
        tr = check(m, x0, step, prec, rounding, True, seed=3, g=5)
        assert tr["t"] > 0
    tel = P.telegraph(0.5, 0.5, 20.0, 1.0)
    check(tel, P.TELEGRAPH_X0, 57, prec, rounding, False, seed=4, g=99)
    bd = P.birth_death()
    check(bd, [0], 0, prec, rounding, False, seed=1, g=0)     # X = 0: the decay channel is zero
    check(bd, [0], 300, prec, rounding, False, seed=1, g=0)


@pytest.mark.parametrize("plant", ["half", "factor_order", "sum_slot", "target_u2"])
def test_recomputation_detects_planted_mistakes(plant):
    """The comparison is sharp enough to see plausible mistakes in either
    implementation: each one planted in the recomputation (standing in for
    the same mistake in the oracle) breaks agreement on the rounding Schloegl
    chain (uniform bfloat16 with SR at X = 560) for some of a few ids."""
    m, x0 = _schlogl_at(560)
    keys = ("a", "S", "E", "U2", "tau", "target", "t_new")
    broke = False
    for g in range(6):
        tr = oracle.trace_step(m, x0, 0, "uniform_bf16", "sr", True, seed=17, g=g)
        good = recompute_step(m, x0, tr["x"], tr["t"], 0, g, 17, "uniform_bf16", "sr", True)
        bad = recompute_step(m, x0, tr["x"], tr["t"], 0, g, 17, "uniform_bf16", "sr", True, plant=plant)
        assert all(np.array_equal(np.asarray(tr[k]), np.asarray(good[k])) for k in keys)
        broke = broke or not all(np.array_equal(np.asarray(tr[k]), np.asarray(bad[k])) for k in keys)
    assert broke, plant
